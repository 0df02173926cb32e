"""Checkpoint files and the resume rule (host code of the library and the
binding; no GPU needed): round trip, rejection of corrupted, truncated or
foreign files and of a file replaced between the header read and the array
read, the mesh and data hashes, and which modes a resumed run may reuse."""
import numpy as np
import pytest

from paper_2009_06725_gb300 import scvs
from synthetic import meshes


def _case(tmp_path, m=3, seed=0):
    mesh = meshes.channel2d(4, 2)
    N, P, d = mesh["xyz"].shape[0], mesh["n_vertices"], 2
    rng = np.random.default_rng(seed)
    u = rng.standard_normal((m, N, d)) + 1j * rng.standard_normal((m, N, d))
    p = rng.standard_normal((m, P)) + 1j * rng.standard_normal((m, P))
    om = 2 * np.pi * np.arange(m)
    st = np.array([scvs.SCVS_CONVERGED, scvs.SCVS_MAX_ITER, scvs.SCVS_CONVERGED][:m], dtype=np.int32)
    rr = np.array([3e-9, 2e-3, 7e-9][:m])
    g = rng.standard_normal((m, 6, d)) + 1j * rng.standard_normal((m, 6, d))
    dh = scvs.mode_data_hashes(g)
    hdr = scvs.scvs_ckpt_header(d, m, N, P, scvs.scvs_mesh_hash(mesh), 1e-8, 1.0, 0.01)
    path = tmp_path / "modes.ckpt"
    scvs.scvs_checkpoint_write(path, hdr, om, dh, st, rr, u, p)
    return mesh, hdr, om, st, rr, u, p, path, g, dh


def test_round_trip(tmp_path):
    mesh, hdr, om, st, rr, u, p, path, g, dh = _case(tmp_path)
    h, om2, dh2, st2, rr2, u2, p2 = scvs.scvs_checkpoint_read(path)
    assert (h.dim, h.n_modes, h.n_nodes, h.n_vertices, h.mesh_hash, h.tol, h.rho, h.mu) == \
        (hdr.dim, hdr.n_modes, hdr.n_nodes, hdr.n_vertices, hdr.mesh_hash, hdr.tol, hdr.rho, hdr.mu)
    for a, b in ((om, om2), (dh, dh2), (st, st2), (rr, rr2), (u, u2), (p, p2)):
        assert np.array_equal(a, b)


def test_file_replaced_between_reads_is_rejected(tmp_path):
    """The array read checks the file against the header the arrays were sized
    for: a larger file swapped in after the header read is refused, not copied."""
    mesh, hdr, om, st, rr, u, p, path, g, dh = _case(tmp_path, m=2)
    h = scvs.scvs_ckpt_header()
    assert scvs.lib().scvs_checkpoint_read(bytes(path), scvs.C.byref(h), None, None, None, None, None, None) == 0
    _case(tmp_path, m=3)  # the same path now holds three modes
    m = h.n_modes
    om2, dh2 = np.zeros(m), np.zeros(m, dtype=np.uint64)
    st2, rr2 = np.zeros(m, dtype=np.int32), np.zeros(m)
    u2 = np.zeros((m, h.n_nodes, h.dim), dtype=np.complex128)
    p2 = np.zeros((m, h.n_vertices), dtype=np.complex128)
    rc = scvs.lib().scvs_checkpoint_read(bytes(path), scvs.C.byref(h), scvs._ptr(om2), scvs._ptr(dh2), scvs._ptr(st2),
                                         scvs._ptr(rr2), scvs._ptr(u2), scvs._ptr(p2))
    assert rc == scvs.SCVS_ERR_ARG and h.n_modes == 2 and not u2.any()


def test_corrupted_truncated_and_foreign_files_are_rejected(tmp_path):
    path = _case(tmp_path)[7]
    raw = bytearray(path.read_bytes())
    bad = tmp_path / "bad.ckpt"
    flipped = bytearray(raw)
    flipped[len(raw) // 2] ^= 0x10  # one bit of the payload
    for data in (bytes(flipped), bytes(raw[:-9]), bytes(raw) + b"x", b"NOTACKPT" + bytes(raw[8:])):
        bad.write_bytes(data)
        with pytest.raises(scvs.ScvsError):
            scvs.scvs_checkpoint_read(bad)
    with pytest.raises(scvs.ScvsError):
        scvs.scvs_checkpoint_read(tmp_path / "missing.ckpt")


def test_mesh_hash_is_deterministic_and_sensitive():
    a, b = meshes.channel2d(4, 2), meshes.channel2d(4, 2)
    assert scvs.scvs_mesh_hash(a) == scvs.scvs_mesh_hash(b)
    tag = b["tag"].copy()
    tag[5] ^= meshes.OUTLET
    assert scvs.scvs_mesh_hash(dict(b, tag=tag)) != scvs.scvs_mesh_hash(a)
    xyz = b["xyz"].copy()
    xyz[7, 1] += 1e-12
    assert scvs.scvs_mesh_hash(dict(b, xyz=xyz)) != scvs.scvs_mesh_hash(a)
    assert scvs.scvs_mesh_hash(meshes.channel2d(4, 3)) != scvs.scvs_mesh_hash(a)


def test_resumable_modes_rule(tmp_path):
    mesh, hdr, om, st, rr, u, p, path, g, dh = _case(tmp_path)
    h, om2, dh2, st2, _, _, _ = scvs.scvs_checkpoint_read(path)
    hsh = scvs.scvs_mesh_hash(mesh)
    # same omegas, reordered and with one new mode; mode 1 of the file did not converge
    cur = np.array([om[2], om[1], 5.0, om[0]])
    cdh = np.array([dh[2], dh[1], 7, dh[0]], dtype=np.uint64)
    assert scvs.resumable_modes(h, om2, dh2, st2, cur, cdh, 1e-8, hsh, 1.0, 0.01).tolist() == [2, -1, -1, 0]
    # a looser tolerance than requested, another mesh or other physics: nothing is reused
    assert scvs.resumable_modes(h, om2, dh2, st2, cur, cdh, 1e-10, hsh, 1.0, 0.01).tolist() == [-1] * 4
    assert scvs.resumable_modes(h, om2, dh2, st2, cur, cdh, 1e-8, hsh ^ 1, 1.0, 0.01).tolist() == [-1] * 4
    assert scvs.resumable_modes(h, om2, dh2, st2, cur, cdh, 1e-8, hsh, 1.0, 0.02).tolist() == [-1] * 4
    assert scvs.resumable_modes(h, om2, dh2, st2, cur, cdh, 1e-8, hsh, 2.0, 0.01).tolist() == [-1] * 4
    # other boundary data for mode 0 (same omega): that mode starts afresh
    g2 = g.copy()
    g2[0, 1, 0] += 1e-9
    cdh2 = scvs.mode_data_hashes(g2)[[2, 1, 1, 0]]
    assert scvs.resumable_modes(h, om2, dh2, st2, cur, cdh2, 1e-8, hsh, 1.0, 0.01).tolist() == [2, -1, -1, -1]


def test_data_hash_sees_dirichlet_and_traction_data():
    g = np.arange(12, dtype=np.complex128).reshape(6, 2)
    h = np.ones((5, 2), dtype=np.complex128)
    base = scvs.scvs_data_hash(g)
    assert scvs.scvs_data_hash(g.copy()) == base
    assert scvs.scvs_data_hash(g, h) != base
    h2 = h.copy()
    h2[3, 1] = 1j
    assert scvs.scvs_data_hash(g, h2) != scvs.scvs_data_hash(g, h)


def test_write_checks_sizes(tmp_path):
    mesh, hdr, om, st, rr, u, p, _, g, dh = _case(tmp_path)
    with pytest.raises(scvs.ScvsError):
        scvs.scvs_checkpoint_write(tmp_path / "x.ckpt", hdr, om, dh, st, rr, u[:, :-1], p)
    bad = scvs.scvs_ckpt_header(4, hdr.n_modes, hdr.n_nodes, hdr.n_vertices, hdr.mesh_hash, hdr.tol, 1.0, 0.01)
    with pytest.raises(scvs.ScvsError):
        scvs.scvs_checkpoint_write(tmp_path / "y.ckpt", bad, om, dh, st, rr, u, p)


def test_modes_to_keep_rule():
    """The a posteriori mode count through the C ABI (host only)."""
    # increments of a k^-2 spectrum: delta_N^2 = E_N / sum_{k<=N} E_k, decreasing
    E = np.array([1.0] + [0.5 * k ** -4.0 for k in range(1, 10)])
    inc = E / np.cumsum(E)
    for eps in (1e-1, 3e-2, 1e-2):  # first reached at N = 3, 5, 8
        n = scvs.scvs_modes_to_keep(inc, eps, patience=1)
        assert np.sqrt(inc[n]) < eps and all(np.sqrt(inc[1:n]) >= eps)
        # with monotone increments a longer patience stops at the same mode
        assert scvs.scvs_modes_to_keep(inc, eps, patience=2) == n
    assert scvs.scvs_modes_to_keep(inc, 1e-12) == 10  # none small enough: keep all
    # a missing harmonic (zero change) followed by an energetic mode
    assert scvs.scvs_modes_to_keep([1.0, 0.0, 0.3], 1e-3, patience=1) == 1
    assert scvs.scvs_modes_to_keep([1.0, 0.0, 0.3], 1e-3) == 3
    assert scvs.scvs_modes_to_keep([1.0, 0.0, 0.3, 0.0, 0.0, 0.2], 1e-3) == 3
    # the last change alone cannot be confirmed by a second one: keep every mode
    assert scvs.scvs_modes_to_keep([1.0, 0.5, 1e-9], 1e-3) == 3
    assert scvs.scvs_modes_to_keep([1.0], 1e-3) == 1
    with pytest.raises(scvs.ScvsError):
        scvs.scvs_modes_to_keep([1.0, 0.1], 0.0)
    with pytest.raises(scvs.ScvsError):
        scvs.scvs_modes_to_keep([1.0, 0.1], 1e-3, patience=0)
