"""Checkpoint files and the resume rule (host code of the library and the
binding; no GPU needed): round trip, rejection of corrupted, truncated or
foreign files, the mesh hash, and which modes a resumed run may reuse."""
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
    hdr = scvs.scvs_ckpt_header(d, m, N, P, scvs.scvs_mesh_hash(mesh), 1e-8)
    path = tmp_path / "modes.ckpt"
    scvs.scvs_checkpoint_write(path, hdr, om, st, rr, u, p)
    return mesh, hdr, om, st, rr, u, p, path


def test_round_trip(tmp_path):
    mesh, hdr, om, st, rr, u, p, path = _case(tmp_path)
    h, om2, st2, rr2, u2, p2 = scvs.scvs_checkpoint_read(path)
    assert (h.dim, h.n_modes, h.n_nodes, h.n_vertices, h.mesh_hash, h.tol) == \
        (hdr.dim, hdr.n_modes, hdr.n_nodes, hdr.n_vertices, hdr.mesh_hash, hdr.tol)
    for a, b in ((om, om2), (st, st2), (rr, rr2), (u, u2), (p, p2)):
        assert np.array_equal(a, b)


def test_corrupted_truncated_and_foreign_files_are_rejected(tmp_path):
    _, _, _, _, _, _, _, path = _case(tmp_path)
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
    mesh, hdr, om, st, rr, u, p, path = _case(tmp_path)
    h, om2, st2, _, _, _ = scvs.scvs_checkpoint_read(path)
    hsh = scvs.scvs_mesh_hash(mesh)
    # same omegas, reordered and with one new mode; mode 1 of the file did not converge
    cur = np.array([om[2], om[1], 5.0, om[0]])
    assert scvs.resumable_modes(h, om2, st2, cur, 1e-8, hsh).tolist() == [2, -1, -1, 0]
    # a looser tolerance than requested, or another mesh: nothing is reused
    assert scvs.resumable_modes(h, om2, st2, cur, 1e-10, hsh).tolist() == [-1] * 4
    assert scvs.resumable_modes(h, om2, st2, cur, 1e-8, hsh ^ 1).tolist() == [-1] * 4


def test_write_checks_sizes(tmp_path):
    mesh, hdr, om, st, rr, u, p, _ = _case(tmp_path)
    with pytest.raises(scvs.ScvsError):
        scvs.scvs_checkpoint_write(tmp_path / "x.ckpt", hdr, om, st, rr, u[:, :-1], p)
    bad = scvs.scvs_ckpt_header(4, hdr.n_modes, hdr.n_nodes, hdr.n_vertices, hdr.mesh_hash, hdr.tol)
    with pytest.raises(scvs.ScvsError):
        scvs.scvs_checkpoint_write(tmp_path / "y.ckpt", bad, om, st, rr, u, p)


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
