"""Seeded synthetic inputs (meshes, boundary data, test vectors) shared by the
oracle, the tests and the benchmark.  Holds none of the method's arithmetic."""
