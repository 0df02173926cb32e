"""Thin ctypes binding of the SCVS C ABI (include/scvs.h).

Argument marshalling only: every step of the solver runs in the CUDA kernels
of ``libscvs.so``.  Functions carry the C names; host arrays are numpy arrays
(copied in/out by the library), device arrays are passed as integer device
addresses (for example ``torch.Tensor.data_ptr()``).  There is no fallback:
if the library is missing or fails to load, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libscvs.so")

SCVS_OK = 0
SCVS_ERR_ARG, SCVS_ERR_MESH, SCVS_ERR_PRESSURE_NULLSPACE = -1, -2, -3
SCVS_ERR_OOM, SCVS_ERR_CUDA, SCVS_ERR_STATE, SCVS_ERR_TIMEOUT = -4, -5, -6, -7
SCVS_TAG_WALL, SCVS_TAG_INLET, SCVS_TAG_OUTLET, SCVS_TAG_NEUMANN = 1, 2, 4, 8
SCVS_CONVERGED, SCVS_MAX_ITER, SCVS_STAGNATED, SCVS_NON_FINITE = 0, 1, 2, 3
SCVS_PREC_MIXED, SCVS_PREC_FP64 = 0, 1
SCVS_PC_BLOCK_CHEB, SCVS_PC_BLOCK_DIAG, SCVS_PC_BLOCK_PMG, SCVS_PC_TRI_PMG, SCVS_PC_TRI_PMG_CS = 0, 1, 2, 3, 4
SCVS_PC_AUTO = 5
SCVS_GUESS_ZERO, SCVS_GUESS_MLP, SCVS_GUESS_CURRENT = 0, 1, 2
SCVS_KRYLOV_FGMRES, SCVS_KRYLOV_COCR = 0, 1
SCVS_CSR_S, SCVS_CSR_G, SCVS_CSR_GT, SCVS_CSR_Q = 0, 1, 2, 3
SCVS_KC_COUNT = 11
SCVS_RECON_STATIC_MAX = 8192
SCVS_TUNE_TILES = 5
TUNE_TILES = (1, 2, 4, 8, 16)
STATUS_NAMES = {0: "converged", 1: "max_iter", 2: "stagnated", 3: "non_finite"}


class scvs_ckpt_header(C.Structure):
    _fields_ = [("dim", C.c_int32), ("n_modes", C.c_int32), ("n_nodes", C.c_int64), ("n_vertices", C.c_int64),
                ("mesh_hash", C.c_uint64), ("tol", C.c_double), ("rho", C.c_double), ("mu", C.c_double)]


class scvs_opts(C.Structure):
    _fields_ = [("tol", C.c_double), ("restart", C.c_int32), ("precision", C.c_int32),
                ("precond", C.c_int32), ("cheb_u", C.c_int32), ("cheb_m", C.c_int32),
                ("cheb_l", C.c_int32), ("max_cycles", C.c_int32), ("guess", C.c_int32),
                ("verbose", C.c_int32), ("cheb_c", C.c_int32), ("autotune", C.c_int32), ("stream", C.c_void_p),
                ("schur_agg", C.c_int32), ("stage", C.c_int32), ("krylov", C.c_int32),
                ("inner_max", C.c_int32), ("graphs", C.c_int32), ("lap_size", C.c_int32), ("lap_smooth", C.c_int32),
                ("reserved", C.c_int32)]


class scvs_mode_report(C.Structure):
    _fields_ = [("status", C.c_int32), ("iterations", C.c_int32), ("cycles", C.c_int32),
                ("guess_used", C.c_int32), ("rel_res", C.c_double), ("res0", C.c_double)]


class scvs_train_opts(C.Structure):
    _fields_ = [("n_pod", C.c_int32), ("hidden", C.c_int32), ("steps", C.c_int32), ("batch", C.c_int32),
                ("lr", C.c_double), ("seed", C.c_uint64), ("max_pod_snapshots", C.c_int32),
                ("reserved", C.c_int32)]


class ScvsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"scvs error {code}: {msg}")
        self.code = code


_lib = None

_P = C.c_void_p
_I32, _I64, _D = C.c_int32, C.c_int64, C.c_double
SIGNATURES = {
    "scvs_default_opts": (None, [C.POINTER(scvs_opts)]),
    "scvs_create": (_I32, [C.POINTER(_P), C.POINTER(scvs_opts)]),
    "scvs_destroy": (None, [_P]),
    "scvs_last_error": (C.c_char_p, [_P]),
    "scvs_set_opts": (_I32, [_P, C.POINTER(scvs_opts)]),
    "scvs_set_mesh": (_I32, [_P, _I32, _I64, _I64, _P, _I64, _P, _P]),
    "scvs_set_mesh_dev": (_I32, [_P, _I32, _I64, _I64, _P, _I64, _P, _P]),
    "scvs_clear_meshes": (_I32, [_P]),
    "scvs_set_physics": (_I32, [_P, _I32, _D, _D]),
    "scvs_set_components": (_I32, [_P, _I32, _I32, _P]),
    "scvs_dirichlet_count": (_I32, [_P, _I32, C.POINTER(_I64)]),
    "scvs_set_modes": (_I32, [_P, _I32, _I32, _P, _P]),
    "scvs_set_modes_dev": (_I32, [_P, _I32, _I32, _P, _P]),
    "scvs_solve": (_I32, [_P, _I32, C.POINTER(scvs_mode_report), _I64]),
    "scvs_get_modal": (_I32, [_P, _I32, _P, _P]),
    "scvs_modal_dev": (_I32, [_P, _I32, C.POINTER(_P), C.POINTER(_I64), C.POINTER(_I32)]),
    "scvs_reconstruct": (_I32, [_P, _I32, _I32, _D, _P, _P]),
    "scvs_reconstruct_dev": (_I32, [_P, _I32, _I32, _D, _P, _P]),
    "scvs_reconstruct_dev_static": (_I32, [_P, _I32, _I32, _D, _P, _P]),
    "scvs_csr_size": (_I32, [_P, _I32, _I32, C.POINTER(_I64), C.POINTER(_I64)]),
    "scvs_get_csr": (_I32, [_P, _I32, _I32, _P, _P]),
    "scvs_get_values": (_I32, [_P, _I32, _I32, _P]),
    "scvs_mode_stride": (_I32, [_P, _I32, C.POINTER(_I32)]),
    "scvs_dof_count": (_I32, [_P, _I32, C.POINTER(_I64)]),
    "scvs_apply": (_I32, [_P, _I32, _I32, _P, _P]),
    "scvs_apply_matfree": (_I32, [_P, _I32, _I32, _P, _P]),
    "scvs_rhs_dev": (_I32, [_P, _I32, C.POINTER(_P)]),
    "scvs_apply_precond": (_I32, [_P, _I32, _P, _P]),
    "scvs_launch_count": (_I64, [_P]),
    "scvs_barrier_selftest": (_I32, [_P, _I64, _I32, _I32, C.POINTER(_I32)]),
    "scvs_pool_usage": (_I32, [_P, _I32, C.POINTER(_I64), C.POINTER(_I64), C.POINTER(_I64)]),
    "scvs_default_train_opts": (None, [C.POINTER(scvs_train_opts)]),
    "scvs_guess_add_snapshots": (_I32, [_P, _I32, _P]),
    "scvs_train_guess": (_I32, [_P, C.POINTER(scvs_train_opts), C.POINTER(_D)]),
    "scvs_guess_set_features": (_I32, [_P, _I32, _P]),
    "scvs_guess_info": (_I32, [_P, C.POINTER(_I64), C.POINTER(_I32), C.POINTER(_I32)]),
    "scvs_guess_reset": (_I32, [_P]),
    "scvs_mlp_init": (_I32, [_P, _I32, _I32, _I32, _P]),
    "scvs_mlp_set_params": (_I32, [_P, _P]),
    "scvs_guess_basis": (_I32, [_P, _I32, _I64, _I32, _P]),
    "scvs_guess_coefficients": (_I32, [_P, _I32, _I64, _I32, _P]),
    "scvs_guess_initial": (_I32, [_P, _I32, _I64, _P, _P]),
    "scvs_mlp_num_params": (_I32, [_P, C.POINTER(_I64)]),
    "scvs_mlp_get_params": (_I32, [_P, _P]),
    "scvs_mlp_forward_dev": (_I32, [_P, _P, _I64, _P]),
    "scvs_mlp_gradient_dev": (_I32, [_P, _P, _P, _I64, _P, C.POINTER(_D)]),
    "scvs_mlp_adam_step": (_I32, [_P, _D]),
    "scvs_tuned_shapes": (_I32, [_P, _I32, _P, _P]),
    "scvs_staged_info": (_I32, [_P, _I32, _P, _P]),
    "scvs_staged_blocks": (_I32, [_P, _I32, _P, _P, _P, _P, _P, _P]),
    "scvs_kernel_timers": (_I32, [_P, _I32]),
    "scvs_kernel_times": (_I32, [_P, _I32, _P, _P, _P]),
    "scvs_set_neumann": (_I32, [_P, _I32, _P, C.POINTER(_I64)]),
    "scvs_bc_spectrum": (_I32, [_P, _I32, _I64, _I32, _P, _P, _P, _P]),
    "scvs_mode_energies": (_I32, [_P, _I32, _I64, _P, _P]),
    "scvs_modes_to_keep": (_I32, [_P, _I64, _D, _I32, C.POINTER(_I64)]),
    "scvs_set_solution": (_I32, [_P, _I32, _P, _P]),
    "scvs_mesh_hash": (_I32, [_I32, _I64, _I64, _P, _I64, _P, _P, C.POINTER(C.c_uint64)]),
    "scvs_checkpoint_write": (_I32, [C.c_char_p, C.POINTER(scvs_ckpt_header), _P, _P, _P, _P, _P, _P]),
    "scvs_checkpoint_read": (_I32, [C.c_char_p, C.POINTER(scvs_ckpt_header), _P, _P, _P, _P, _P, _P]),
    "scvs_data_hash": (_I32, [_P, _I64, _P, _I64, C.POINTER(C.c_uint64)]),
    "scvs_graph_aggregates": (_I32, [_I64, _P, _P, _I32, _P, C.POINTER(_I32), C.POINTER(_I32)]),
    "scvs_schur_coarse_info": (_I32, [_P, _I32, _P]),
    "scvs_lap_info": (_I32, [_P, _I32, _P, _P]),
    "scvs_pc_bounds": (_I32, [_P, _I32, _I32, _P]),
}
KERNEL_CLASSES = ["spmm_fp32", "spmm_fp64", "precond", "arnoldi", "vector", "assembly", "reconstruct", "matfree",
                  "cheb_fine", "pressure", "coarse"]


def lib():
    """Load libscvs.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} not built: run paper_2009_06725_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _check(ctx, rc):
    if rc < 0:
        msg = lib().scvs_last_error(ctx)
        raise ScvsError(rc, msg.decode() if msg else "")
    return rc


def scvs_default_opts(**overrides):
    o = scvs_opts()
    lib().scvs_default_opts(C.byref(o))
    for k, v in overrides.items():
        setattr(o, k, v)
    return o


def scvs_create(opts=None):
    h = C.c_void_p()
    rc = lib().scvs_create(C.byref(h), C.byref(opts) if opts is not None else None)
    if rc < 0:
        raise ScvsError(rc, "scvs_create failed")
    return h


def scvs_destroy(ctx):
    lib().scvs_destroy(ctx)


def scvs_last_error(ctx):
    return lib().scvs_last_error(ctx).decode()


def scvs_set_opts(ctx, opts):
    return _check(ctx, lib().scvs_set_opts(ctx, C.byref(opts)))


def scvs_set_mesh(ctx, mesh):
    """mesh: dict with dim, xyz float64 [N][d], conn int32 [E][nl], tag uint8 [N], n_vertices."""
    xyz = np.ascontiguousarray(mesh["xyz"], dtype=np.float64)
    conn = np.ascontiguousarray(mesh["conn"], dtype=np.int32)
    tag = np.ascontiguousarray(mesh["tag"], dtype=np.uint8)
    return _check(ctx, lib().scvs_set_mesh(ctx, int(mesh["dim"]), xyz.shape[0], int(mesh["n_vertices"]),
                                           _ptr(xyz), conn.shape[0], _ptr(conn), _ptr(tag)))


def scvs_set_mesh_dev(ctx, dim, n_nodes, n_vertices, xyz_dev, n_elem, conn_dev, tag_dev):
    return _check(ctx, lib().scvs_set_mesh_dev(ctx, dim, n_nodes, n_vertices, xyz_dev, n_elem, conn_dev, tag_dev))


def scvs_clear_meshes(ctx):
    return _check(ctx, lib().scvs_clear_meshes(ctx))


def scvs_set_components(ctx, mesh_id, n_comp, node_comp):
    nc = np.ascontiguousarray(node_comp, dtype=np.int32)
    return _check(ctx, lib().scvs_set_components(ctx, mesh_id, n_comp, _ptr(nc)))


def scvs_set_physics(ctx, mesh_id, rho, mu):
    return _check(ctx, lib().scvs_set_physics(ctx, mesh_id, rho, mu))


def scvs_dirichlet_count(ctx, mesh_id):
    n = C.c_int64()
    _check(ctx, lib().scvs_dirichlet_count(ctx, mesh_id, C.byref(n)))
    return n.value


def scvs_set_modes(ctx, mesh_id, omega, g):
    """omega float64 [m]; g complex128 [m][n_dir][dim]."""
    om = np.ascontiguousarray(omega, dtype=np.float64)
    gg = np.ascontiguousarray(g, dtype=np.complex128)
    return _check(ctx, lib().scvs_set_modes(ctx, mesh_id, om.size, _ptr(om), _ptr(gg)))


def scvs_set_modes_dev(ctx, mesh_id, omega, g_dev):
    om = np.ascontiguousarray(omega, dtype=np.float64)
    return _check(ctx, lib().scvs_set_modes_dev(ctx, mesh_id, om.size, _ptr(om), g_dev))


def scvs_solve(ctx, mesh_id=-1, n_reports=0):
    """Returns a list of dicts (status, iterations, cycles, rel_res, guess_used, res0)."""
    rep = (scvs_mode_report * max(1, n_reports))()
    _check(ctx, lib().scvs_solve(ctx, mesh_id, rep, n_reports))
    return [dict(status=r.status, iterations=r.iterations, cycles=r.cycles, rel_res=r.rel_res,
                 guess_used=r.guess_used, res0=r.res0) for r in rep[:n_reports]]


def _out(shape, dtype, out):
    """Caller-provided output array (e.g. a pinned-memory view), checked, or a new one."""
    if out is None:
        return np.empty(shape, dtype=dtype)
    if out.shape != tuple(shape) or out.dtype != dtype or not out.flags.c_contiguous or not out.flags.writeable:
        raise ValueError(f"output array must be a writeable C-contiguous {np.dtype(dtype).name} array of shape {shape}")
    return out


def scvs_get_modal(ctx, mesh_id, n_modes, n_nodes, dim, n_vertices, out_u=None, out_p=None):
    u = _out((n_modes, n_nodes, dim), np.complex128, out_u)
    p = _out((n_modes, n_vertices), np.complex128, out_p)
    _check(ctx, lib().scvs_get_modal(ctx, mesh_id, _ptr(u), _ptr(p)))
    return u, p


def scvs_modal_dev(ctx, mesh_id):
    x = C.c_void_p()
    n = C.c_int64()
    ld = C.c_int32()
    _check(ctx, lib().scvs_modal_dev(ctx, mesh_id, C.byref(x), C.byref(n), C.byref(ld)))
    return x.value, n.value, ld.value


def scvs_reconstruct(ctx, mesh_id, n_t, period, n_nodes, dim, n_vertices, out_u=None, out_p=None):
    u = _out((n_t, n_nodes, dim), np.float64, out_u)
    p = _out((n_t, n_vertices), np.float64, out_p)
    _check(ctx, lib().scvs_reconstruct(ctx, mesh_id, n_t, period, _ptr(u), _ptr(p)))
    return u, p


def scvs_reconstruct_dev(ctx, mesh_id, n_t, period, u_dev, p_dev):
    return _check(ctx, lib().scvs_reconstruct_dev(ctx, mesh_id, n_t, period, u_dev, p_dev))


def scvs_reconstruct_dev_static(ctx, mesh_id, n_t, period, u_dev, p_dev):
    """Allocation-free reconstruction (static twiddle table; see include/scvs.h)."""
    return _check(ctx, lib().scvs_reconstruct_dev_static(ctx, mesh_id, n_t, period, u_dev, p_dev))


def scvs_csr_size(ctx, mesh_id, which):
    r, z = C.c_int64(), C.c_int64()
    _check(ctx, lib().scvs_csr_size(ctx, mesh_id, which, C.byref(r), C.byref(z)))
    return r.value, z.value


def scvs_get_csr(ctx, mesh_id, which):
    nr, nnz = scvs_csr_size(ctx, mesh_id, which)
    rowptr = np.empty(nr + 1, dtype=np.int64)
    col = np.empty(max(nnz, 1), dtype=np.int32)
    _check(ctx, lib().scvs_get_csr(ctx, mesh_id, which, _ptr(rowptr), _ptr(col)))
    return rowptr, col[:nnz]


def scvs_get_values(ctx, mesh_id, which, dim):
    _, nnz = scvs_csr_size(ctx, mesh_id, which)
    rows = 2 if which in (SCVS_CSR_S, SCVS_CSR_Q) else dim
    v = np.empty((rows, max(nnz, 1)), dtype=np.float64)
    _check(ctx, lib().scvs_get_values(ctx, mesh_id, which, _ptr(v)))
    return v[:, :nnz]


def scvs_mode_stride(ctx, mesh_id):
    ld = C.c_int32()
    _check(ctx, lib().scvs_mode_stride(ctx, mesh_id, C.byref(ld)))
    return ld.value


def scvs_dof_count(ctx, mesh_id):
    n = C.c_int64()
    _check(ctx, lib().scvs_dof_count(ctx, mesh_id, C.byref(n)))
    return n.value


def scvs_apply(ctx, mesh_id, precision, x_dev, y_dev):
    return _check(ctx, lib().scvs_apply(ctx, mesh_id, precision, x_dev, y_dev))


def scvs_apply_matfree(ctx, mesh_id, precision, x_dev, y_dev):
    return _check(ctx, lib().scvs_apply_matfree(ctx, mesh_id, precision, x_dev, y_dev))


def scvs_rhs_dev(ctx, mesh_id):
    b = C.c_void_p()
    _check(ctx, lib().scvs_rhs_dev(ctx, mesh_id, C.byref(b)))
    return b.value


def scvs_apply_precond(ctx, mesh_id, r_dev, z_dev):
    return _check(ctx, lib().scvs_apply_precond(ctx, mesh_id, r_dev, z_dev))


def scvs_launch_count(ctx):
    return lib().scvs_launch_count(ctx)


def scvs_barrier_selftest(ctx, spin_limit, n_blocks, absent_block):
    """Bounded grid-barrier self-test: returns (status code, blocks passed);
    SCVS_ERR_TIMEOUT is returned, not raised."""
    n = C.c_int32(0)
    rc = lib().scvs_barrier_selftest(ctx, int(spin_limit), int(n_blocks), int(absent_block), C.byref(n))
    if rc < 0 and rc != SCVS_ERR_TIMEOUT:
        _check(ctx, rc)
    return rc, n.value


def scvs_pool_usage(ctx, reset_high=False):
    """(used, used_high, reserved) bytes of the context's device memory pool;
    reset_high then resets the high-water mark to the current use."""
    u, h, r = C.c_int64(), C.c_int64(), C.c_int64()
    _check(ctx, lib().scvs_pool_usage(ctx, 1 if reset_high else 0, C.byref(u), C.byref(h), C.byref(r)))
    return u.value, h.value, r.value


def scvs_default_train_opts(**overrides):
    o = scvs_train_opts()
    lib().scvs_default_train_opts(C.byref(o))
    for k, v in overrides.items():
        setattr(o, k, v)
    return o


def scvs_guess_add_snapshots(ctx, mesh_id, features):
    f = np.ascontiguousarray(features, dtype=np.float64)
    return _check(ctx, lib().scvs_guess_add_snapshots(ctx, mesh_id, _ptr(f)))


def scvs_train_guess(ctx, opts=None):
    loss = C.c_double()
    _check(ctx, lib().scvs_train_guess(ctx, C.byref(opts) if opts is not None else None, C.byref(loss)))
    return loss.value


def scvs_guess_set_features(ctx, mesh_id, features):
    f = np.ascontiguousarray(features, dtype=np.float64)
    return _check(ctx, lib().scvs_guess_set_features(ctx, mesh_id, _ptr(f)))


def scvs_guess_info(ctx):
    n, r, t = C.c_int64(), C.c_int32(), C.c_int32()
    _check(ctx, lib().scvs_guess_info(ctx, C.byref(n), C.byref(r), C.byref(t)))
    return dict(n_snapshots=n.value, n_pod=r.value, trained=bool(t.value))


def scvs_guess_reset(ctx):
    return _check(ctx, lib().scvs_guess_reset(ctx))


def scvs_mlp_init(ctx, n_in, hidden, n_out, params):
    p = np.ascontiguousarray(params, dtype=np.float32)
    return _check(ctx, lib().scvs_mlp_init(ctx, n_in, hidden, n_out, _ptr(p)))


def scvs_mlp_set_params(ctx, params):
    p = np.ascontiguousarray(params, dtype=np.float32)
    return _check(ctx, lib().scvs_mlp_set_params(ctx, _ptr(p)))


def scvs_guess_basis(ctx, block, n_rows):
    """POD basis of block 0 (velocity) or 1 (pressure): complex [n_rows][n_pod]."""
    r = scvs_guess_info(ctx)["n_pod"]
    out = np.empty((n_rows, r), dtype=np.complex128)
    _check(ctx, lib().scvs_guess_basis(ctx, block, n_rows, r, _ptr(out)))
    return out


def scvs_guess_coefficients(ctx, block):
    """POD coefficients of the training snapshots: complex [n_snapshots][n_pod]."""
    info = scvs_guess_info(ctx)
    out = np.empty((info["n_snapshots"], info["n_pod"]), dtype=np.complex128)
    _check(ctx, lib().scvs_guess_coefficients(ctx, block, info["n_snapshots"], info["n_pod"], _ptr(out)))
    return out


def scvs_guess_initial(ctx, mesh_id, n_modes):
    """Learned start of every mode without solving: (res0 [m], kept [m] bool);
    x0 is left as the mesh's solution (read it with scvs_get_modal)."""
    res0 = np.empty(n_modes, dtype=np.float64)
    kept = np.empty(n_modes, dtype=np.int32)
    _check(ctx, lib().scvs_guess_initial(ctx, mesh_id, n_modes, _ptr(res0), _ptr(kept)))
    return res0, kept.astype(bool)


def scvs_mlp_num_params(ctx):
    n = C.c_int64()
    _check(ctx, lib().scvs_mlp_num_params(ctx, C.byref(n)))
    return n.value


def scvs_mlp_get_params(ctx):
    out = np.empty(scvs_mlp_num_params(ctx), dtype=np.float32)
    _check(ctx, lib().scvs_mlp_get_params(ctx, _ptr(out)))
    return out


def scvs_mlp_forward_dev(ctx, x_dev, batch, y_dev):
    return _check(ctx, lib().scvs_mlp_forward_dev(ctx, x_dev, batch, y_dev))


def scvs_mlp_gradient_dev(ctx, x_dev, t_dev, batch):
    g = np.empty(scvs_mlp_num_params(ctx), dtype=np.float32)
    loss = C.c_double()
    _check(ctx, lib().scvs_mlp_gradient_dev(ctx, x_dev, t_dev, batch, _ptr(g), C.byref(loss)))
    return g, loss.value


def scvs_mlp_adam_step(ctx, lr):
    return _check(ctx, lib().scvs_mlp_adam_step(ctx, lr))


def scvs_staged_info(ctx, mesh_id):
    """Row blocks and staged-gather choice of a mesh (see include/scvs.h)."""
    info = np.zeros(10, dtype=np.int64)
    us = np.zeros(8, dtype=np.float32)
    _check(ctx, lib().scvs_staged_info(ctx, mesh_id, _ptr(info), _ptr(us)))
    keys = ("valid", "n_blk", "budget", "fp_max", "fv_max", "fp_total", "st_spmm", "st_cheb", "runs_spmm",
            "runs_cheb")
    out = {k: int(v) for k, v in zip(keys, info)}
    for k in ("valid", "runs_spmm", "runs_cheb"):
        out[k] = bool(out[k])
    out["spmm_us"] = [float(v) for v in us[:4]]
    out["cheb_us"] = [float(v) for v in us[4:]]
    return out


def scvs_staged_blocks(ctx, mesh_id, n_nodes, s_nnz):
    """Host copies of the row blocks: perm, row0, fp_ptr, fp_col, fv_len, lcol."""
    info = scvs_staged_info(ctx, mesh_id)
    nb = info["n_blk"]
    perm = np.empty(n_nodes, dtype=np.int32)
    row0 = np.empty(nb + 1, dtype=np.int64)
    fp_ptr = np.empty(nb + 1, dtype=np.int64)
    fp_col = np.empty(max(info["fp_total"], 1), dtype=np.int32)
    fv_len = np.empty(nb, dtype=np.int32)
    lcol = np.empty(s_nnz, dtype=np.uint16)
    _check(ctx, lib().scvs_staged_blocks(ctx, mesh_id, _ptr(perm), _ptr(row0), _ptr(fp_ptr), _ptr(fp_col),
                                         _ptr(fv_len), _ptr(lcol)))
    return dict(perm=perm, row0=row0, fp_ptr=fp_ptr, fp_col=fp_col[:info["fp_total"]], fv_len=fv_len, lcol=lcol)


def scvs_tuned_shapes(ctx, mesh_id):
    """Autotuned launch shapes of a mesh and the candidate times (us) as
    {kernel: [[t(mpl, tile) for tile in TUNE_TILES] for mpl in (1, 2, 4)]}."""
    shape = np.zeros(4, dtype=np.int32)
    nt = len(TUNE_TILES)
    us = np.zeros(2 * 3 * nt, dtype=np.float32)
    _check(ctx, lib().scvs_tuned_shapes(ctx, mesh_id, _ptr(shape), _ptr(us)))
    us = us.reshape(2, 3, nt).round(1).tolist()
    return dict(mpl_spmm=int(shape[0]), tile_spmm=int(shape[1]), mpl_cheb=int(shape[2]), tile_cheb=int(shape[3]),
                spmm_us=us[0], cheb_us=us[1])


def scvs_set_neumann(ctx, mesh_id, h):
    """Nodal tractions h [n_modes][n_nodes][dim] (complex) on the faces tagged
    SCVS_TAG_NEUMANN; returns the number of such faces."""
    hh = np.ascontiguousarray(h, dtype=np.complex128)
    nf = C.c_int64(0)
    _check(ctx, lib().scvs_set_neumann(ctx, mesh_id, _ptr(hh), C.byref(nf)))
    return nf.value


def scvs_bc_spectrum(ctx, g_t_dev, n_t, n_pts, n_modes, c_dev, w_dev=None):
    """Per-mode data c [n_modes][n_pts] (complex128, written to device memory
    at c_dev) of the device samples g_t_dev [n_t][n_pts] (FP64) and the
    truncation errors e2 [n_modes] (numpy)."""
    e2 = np.zeros(n_modes)
    _check(ctx, lib().scvs_bc_spectrum(ctx, n_t, n_pts, n_modes, g_t_dev, w_dev, c_dev, _ptr(e2)))
    return e2


def scvs_mode_energies(ctx, mesh_id, n_out):
    """(E, incr2), each [n_out] = [n_components * n_modes]: time-averaged L2 energy of every
    solved mode's velocity and the a posteriori increments of the truncated reconstruction."""
    E = np.zeros(n_out)
    inc = np.zeros(n_out)
    _check(ctx, lib().scvs_mode_energies(ctx, mesh_id, n_out, _ptr(E), _ptr(inc)))
    return E, inc


def scvs_set_solution(ctx, mesh_id, u, p):
    """Initial solution [n_modes][N][d], [n_modes][P] (complex) for opts.guess = SCVS_GUESS_CURRENT."""
    uu = np.ascontiguousarray(u, dtype=np.complex128)
    pp = np.ascontiguousarray(p, dtype=np.complex128)
    return _check(ctx, lib().scvs_set_solution(ctx, mesh_id, _ptr(uu), _ptr(pp)))


def scvs_mesh_hash(mesh):
    """FNV-1a 64 hash of a mesh dict's arrays (host only)."""
    xyz = np.ascontiguousarray(mesh["xyz"], dtype=np.float64)
    conn = np.ascontiguousarray(mesh["conn"], dtype=np.int32)
    tag = np.ascontiguousarray(mesh["tag"], dtype=np.uint8)
    h = C.c_uint64(0)
    rc = lib().scvs_mesh_hash(mesh["dim"], xyz.shape[0], mesh["n_vertices"], _ptr(xyz), conn.shape[0], _ptr(conn),
                              _ptr(tag), C.byref(h))
    if rc < 0:
        raise ScvsError(rc, "scvs_mesh_hash: bad mesh")
    return h.value


def scvs_data_hash(g, h=None):
    """FNV-1a 64 hash of one mode's boundary data (Dirichlet values, optional tractions)."""
    ga = np.ascontiguousarray(g, dtype=np.complex128).ravel()
    ha = None if h is None else np.ascontiguousarray(h, dtype=np.complex128).ravel()
    out = C.c_uint64()
    rc = lib().scvs_data_hash(_ptr(ga), ga.size, _ptr(ha), 0 if ha is None else ha.size, C.byref(out))
    if rc < 0:
        raise ScvsError(rc, "scvs_data_hash: bad argument")
    return out.value


def scvs_checkpoint_write(path, header, omega, data_hash, status, rel_res, u, p):
    arrs = [np.ascontiguousarray(omega, dtype=np.float64), np.ascontiguousarray(data_hash, dtype=np.uint64),
            np.ascontiguousarray(status, dtype=np.int32), np.ascontiguousarray(rel_res, dtype=np.float64),
            np.ascontiguousarray(u, dtype=np.complex128), np.ascontiguousarray(p, dtype=np.complex128)]
    m = header.n_modes
    shapes = [(m,), (m,), (m,), (m,), (m, header.n_nodes, header.dim), (m, header.n_vertices)]
    for a, sh in zip(arrs, shapes):
        if a.size != int(np.prod(sh)):
            raise ScvsError(SCVS_ERR_ARG, "scvs_checkpoint_write: array size does not match the header")
    rc = lib().scvs_checkpoint_write(os.fsencode(path), C.byref(header), *[_ptr(a) for a in arrs])
    if rc < 0:
        raise ScvsError(rc, f"scvs_checkpoint_write: cannot write {path}")


def scvs_checkpoint_read(path):
    """(header, omega, data_hash, status, rel_res, u [m][N][d], p [m][P]); raises ScvsError on
    a bad file, or if the file changed between the header read and the array read."""
    h = scvs_ckpt_header()
    rc = lib().scvs_checkpoint_read(os.fsencode(path), C.byref(h), None, None, None, None, None, None)
    if rc < 0:
        raise ScvsError(rc, f"scvs_checkpoint_read: bad checkpoint {path}")
    m = h.n_modes
    om, dh, st, rr = np.zeros(m), np.zeros(m, dtype=np.uint64), np.zeros(m, dtype=np.int32), np.zeros(m)
    u = np.zeros((m, h.n_nodes, h.dim), dtype=np.complex128)
    p = np.zeros((m, h.n_vertices), dtype=np.complex128)
    rc = lib().scvs_checkpoint_read(os.fsencode(path), C.byref(h), _ptr(om), _ptr(dh), _ptr(st), _ptr(rr), _ptr(u),
                                    _ptr(p))
    if rc < 0:
        raise ScvsError(rc, f"scvs_checkpoint_read: bad checkpoint {path}")
    return h, om, dh, st, rr, u, p


def mode_data_hashes(g, h=None):
    """Per-mode boundary-data hashes: g [m][n_dir][d], h [m][N][d] or None."""
    return np.array([scvs_data_hash(g[k], None if h is None else h[k]) for k in range(len(g))], dtype=np.uint64)


def save_checkpoint(ctx, mesh_id, mesh, omegas, reports, tol, path, rho, mu, g, h=None):
    """Write the modal solution of a solved mesh with its per-mode status (a mode counts as
    converged when every component's system of that mode converged), the physics and the
    hash of every mode's boundary data."""
    m = len(omegas)
    N, P, d = mesh["xyz"].shape[0], mesh["n_vertices"], mesh["dim"]
    u, p = scvs_get_modal(ctx, mesh_id, m, N, d, P)
    n_comp = max(1, len(reports) // m)
    status = np.array([SCVS_CONVERGED if all(reports[c * m + k]["status"] == SCVS_CONVERGED for c in range(n_comp))
                       else SCVS_MAX_ITER for k in range(m)], dtype=np.int32)
    rel = np.array([max(reports[c * m + k]["rel_res"] for c in range(n_comp)) for k in range(m)])
    hdr = scvs_ckpt_header(d, m, N, P, scvs_mesh_hash(mesh), float(tol), float(rho), float(mu))
    scvs_checkpoint_write(path, hdr, omegas, mode_data_hashes(g, h), status, rel, u, p)


def resumable_modes(header, f_omega, f_hash, f_status, omegas, data_hash, tol, mesh_hash, rho, mu):
    """For every current mode k, the checkpoint mode j with the same omega and the same
    boundary-data hash (exact) that converged to a tolerance at least as tight on the same
    mesh with the same physics, else -1."""
    out = np.full(len(omegas), -1, dtype=np.int64)
    if header.mesh_hash != mesh_hash or header.tol > tol or header.rho != rho or header.mu != mu:
        return out
    for k, w in enumerate(omegas):
        for j in range(header.n_modes):
            if f_omega[j] == w and int(f_hash[j]) == int(data_hash[k]) and f_status[j] == SCVS_CONVERGED:
                out[k] = j
                break
    return out


def resume_from_checkpoint(ctx, mesh_id, mesh, omegas, tol, path, rho, mu, g, h=None):
    """Load the matching modes of a checkpoint as the initial solution (the others start
    from zero); solve next with opts.guess = SCVS_GUESS_CURRENT.  Returns the map of
    resumable_modes."""
    hd, om, dh, st, _, u, p = scvs_checkpoint_read(path)
    if hd.n_nodes != mesh["xyz"].shape[0] or hd.n_vertices != mesh["n_vertices"] or hd.dim != mesh["dim"]:
        return np.full(len(omegas), -1, dtype=np.int64)
    idx = resumable_modes(hd, om, dh, st, omegas, mode_data_hashes(g, h), tol, scvs_mesh_hash(mesh), rho, mu)
    u0 = np.zeros((len(omegas), hd.n_nodes, hd.dim), dtype=np.complex128)
    p0 = np.zeros((len(omegas), hd.n_vertices), dtype=np.complex128)
    for k, j in enumerate(idx):
        if j >= 0:
            u0[k], p0[k] = u[j], p[j]
    scvs_set_solution(ctx, mesh_id, u0, p0)
    return idx


def scvs_modes_to_keep(incr2, eps, patience=2):
    """A posteriori number of modes (Sec. 3): the smallest N >= 1 whose next
    `patience` reconstruction changes (sqrt of incr2) are all below eps; all
    modes if none."""
    inc = np.ascontiguousarray(incr2, dtype=np.float64)
    n = C.c_int64(0)
    rc = lib().scvs_modes_to_keep(_ptr(inc), inc.size, float(eps), int(patience), C.byref(n))
    if rc < 0:
        raise ScvsError(rc, "scvs_modes_to_keep: bad argument")
    return n.value


def scvs_graph_aggregates(row_ptr, col, target):
    """Graph aggregates of a vertex graph given as CSR (host only).  Returns
    (agg [n] int32, n_agg, n_blk)."""
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    n = row_ptr.size - 1
    agg = np.empty(max(n, 0), dtype=np.int32)
    na, nb = C.c_int32(0), C.c_int32(0)
    rc = lib().scvs_graph_aggregates(n, _ptr(row_ptr), _ptr(col), int(target), _ptr(agg), C.byref(na), C.byref(nb))
    if rc < 0:
        raise ScvsError(rc, "scvs_graph_aggregates: bad argument")
    return agg, na.value, nb.value


def scvs_schur_coarse_info(ctx, mesh_id):
    """{n_agg, n_blk, na_max, singular} of the last coarse Schur setup (zeros before it)."""
    info = np.zeros(4, dtype=np.int32)
    _check(ctx, lib().scvs_schur_coarse_info(ctx, mesh_id, _ptr(info)))
    return dict(n_agg=int(info[0]), n_blk=int(info[1]), na_max=int(info[2]), singular=int(info[3]))


def scvs_lap_info(ctx, mesh_id, n_vertices=None):
    """{on, n_agg, n_blk, na_max, singular, unanchored} of the two-level pressure
    Laplacian's coarse level, plus 'agg' ([n_vertices] int32, -1 on the outlet)
    when n_vertices is given."""
    info = np.zeros(6, dtype=np.int32)
    agg = None if n_vertices is None else np.empty(int(n_vertices), dtype=np.int32)
    _check(ctx, lib().scvs_lap_info(ctx, mesh_id, _ptr(info), None if agg is None else _ptr(agg)))
    out = dict(on=int(info[0]), n_agg=int(info[1]), n_blk=int(info[2]), na_max=int(info[3]),
               singular=int(info[4]), unanchored=int(info[5]))
    if agg is not None:
        out["agg"] = agg
    return out


def scvs_pc_bounds(ctx, mesh_id, n_modes):
    """(lam_m, lam_l, lam_u [n_modes], lam_c [n_modes]): the power-method
    estimates behind the preconditioner's Chebyshev intervals."""
    out = np.empty(2 + 2 * n_modes, dtype=np.float64)
    _check(ctx, lib().scvs_pc_bounds(ctx, mesh_id, int(n_modes), _ptr(out)))
    return float(out[0]), float(out[1]), out[2:2 + n_modes].copy(), out[2 + n_modes:].copy()


def scvs_kernel_timers(ctx, enable):
    return _check(ctx, lib().scvs_kernel_timers(ctx, 1 if enable else 0))


def scvs_kernel_times(ctx):
    """{class: (ms, algorithmic bytes, launches)} summed since the timers were enabled."""
    n = len(KERNEL_CLASSES)
    ms = np.zeros(n)
    by = np.zeros(n)
    ln = np.zeros(n, dtype=np.int64)
    _check(ctx, lib().scvs_kernel_times(ctx, n, _ptr(ms), _ptr(by), _ptr(ln)))
    return {k: (float(ms[i]), float(by[i]), int(ln[i])) for i, k in enumerate(KERNEL_CLASSES)}


class Solver:
    """Convenience owner of one context (closes it on exit)."""

    def __init__(self, **opts):
        self.opts = scvs_default_opts(**opts)
        self.ctx = scvs_create(self.opts)

    def close(self):
        if self.ctx is not None:
            scvs_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_opts(self, **kw):
        for k, v in kw.items():
            setattr(self.opts, k, v)
        scvs_set_opts(self.ctx, self.opts)
