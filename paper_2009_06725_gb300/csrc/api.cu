// C ABI of the SCVS library: argument checking, error mapping, host <-> device
// marshalling.  Every computation runs in the kernels of assembly.cu,
// operators.cu, krylov.cu and recon.cu.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>
#include "scvs_internal.h"
#include "opargs.cuh"

using namespace scvs;

struct scvs_ctx : public Ctx {};

namespace scvs {
void KTimers::begin(cudaStream_t s) {
  if (pool.empty()) {
    cudaEvent_t a, b;
    SCVS_CUDA(cudaEventCreate(&a));
    SCVS_CUDA(cudaEventCreate(&b));
    pool.push_back({a, b});
  }
  cur_a = pool.back().first;
  SCVS_CUDA(cudaEventRecord(cur_a, s));
}
void KTimers::end(cudaStream_t s, int cls, double nbytes) {
  auto pr = pool.back();
  pool.pop_back();
  SCVS_CUDA(cudaEventRecord(pr.second, s));
  pend.push_back({pr.first, pr.second, cls, nbytes});
  if (pend.size() > 4096) resolve();
}
void KTimers::resolve() {
  for (auto &p : pend) {
    SCVS_CUDA(cudaEventSynchronize(p.b));
    float t = 0;
    SCVS_CUDA(cudaEventElapsedTime(&t, p.a, p.b));
    ms[p.cls] += t;
    bytes[p.cls] += p.bytes;
    n[p.cls] += 1;
    pool.push_back({p.a, p.b});
  }
  pend.clear();
}
void KTimers::reset() {
  resolve();
  for (int i = 0; i < KC_COUNT; ++i) { ms[i] = 0; bytes[i] = 0; n[i] = 0; }
}
void KTimers::destroy() {
  for (auto &p : pend) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
  for (auto &p : pool) { cudaEventDestroy(p.first); cudaEventDestroy(p.second); }
  pend.clear();
  pool.clear();
}

int dev_error(Ctx &c) {
  int e = 0;
  SCVS_CUDA(cudaMemcpyAsync(&e, c.dev_err, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
  SCVS_CUDA(cudaStreamSynchronize(c.stream));
  if (e) SCVS_CUDA(cudaMemsetAsync(c.dev_err, 0, sizeof(int), c.stream));
  return e;
}
}  // namespace scvs

namespace {

std::string deverr_text(int bits) {
  std::string s;
  if (bits & DEVERR_BAD_NODE) s += "connectivity entry outside [0, n_nodes) or node unused; ";
  if (bits & DEVERR_BAD_VERTEX) s += "simplex vertex id >= n_vertices or edge node id < n_vertices; ";
  if (bits & DEVERR_JACOBIAN) s += "element with non-positive Jacobian; ";
  if (bits & DEVERR_VALENCE) s += "too many elements around one node; ";
  if (bits & DEVERR_BARRIER) s += "grid barrier timeout; ";
  if (bits & DEVERR_DUP_NODE) s += "element lists a node twice; ";
  return s;
}

template <typename F>
int guarded(scvs_ctx *c, F &&f) {
  if (!c) return SCVS_ERR_ARG;
  try {
    int r = f();
    if (r == SCVS_OK || r >= 0) c->err.clear();
    return r;
  } catch (const CudaError &e) {
    c->err = std::string("CUDA error ") + cudaGetErrorString(e.code) + " in " + e.where;
    (void)cudaGetLastError();
    return SCVS_ERR_CUDA;
  } catch (const std::bad_alloc &) {
    c->err = "device allocation failed";
    return SCVS_ERR_OOM;
  } catch (int code) {
    if (code < 0) {
      if (c->err.empty()) c->err = "error " + std::to_string(code);
      return code;
    }
    c->err = "invalid mesh: " + deverr_text(code);
    return (code & DEVERR_BARRIER) ? SCVS_ERR_TIMEOUT : SCVS_ERR_MESH;
  }
}

int fail(scvs_ctx *c, int code, const std::string &msg) {
  c->err = msg;
  return code;
}

Mesh *get_mesh(scvs_ctx *c, int id) {
  if (id < 0 || id >= (int)c->meshes.size() || !c->meshes[id]) return nullptr;
  return c->meshes[id];
}

int mode_stride(int m) {
  int ld = 2;
  while (ld < m) ld <<= 1;
  return ld;
}

int add_mesh(scvs_ctx *c, int dim, int64_t N, int64_t P, const double *xyz, int64_t E, const int32_t *conn,
             const uint8_t *tag, bool on_device) {
  if (dim != 2 && dim != 3) return fail(c, SCVS_ERR_ARG, "dim must be 2 or 3");
  if (N <= 0 || P <= 0 || P > N || E <= 0) return fail(c, SCVS_ERR_ARG, "bad mesh sizes");
  if (N >= INT32_MAX || E * (dim == 2 ? 6 : 10) >= INT32_MAX) return fail(c, SCVS_ERR_ARG, "mesh too large for int32 ids");
  if (!xyz || !conn || !tag) return fail(c, SCVS_ERR_ARG, "null mesh array");
  std::vector<uint8_t> htag(N);
  SCVS_CUDA(cudaMemcpy(htag.data(), tag, N, on_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost));
  std::vector<int64_t> dn;
  int64_t n_out = 0;
  for (int64_t i = 0; i < N; ++i) {
    if (htag[i] & (SCVS_TAG_WALL | SCVS_TAG_INLET)) dn.push_back(i);
    if (i < P && (htag[i] & SCVS_TAG_OUTLET)) ++n_out;
  }
  if (n_out == 0)
    return fail(c, SCVS_ERR_PRESSURE_NULLSPACE,
                "no vertex tagged OUTLET: with velocity prescribed on the whole boundary the pressure is undetermined");
  Mesh *m = new Mesh();
  m->arena.pool = m->mode_arena.pool = c->pool;
  m->arena.stream = m->mode_arena.stream = c->stream;
  m->dim = dim;
  m->nl = dim == 2 ? 6 : 10;
  m->nv = dim + 1;
  m->N = N; m->P = P; m->E = E;
  m->n_dof = (int64_t)dim * N + P;
  m->n_dir = (int64_t)dn.size();
  try {
    build_mesh(*c, *m, xyz, conn, tag);
    set_chunks(*c, *m, nullptr, 1);
    m->dir_nodes = m->arena.alloc<int64_t>(std::max<int64_t>(1, m->n_dir));
    if (m->n_dir) {
      SCVS_CUDA(cudaMemcpyAsync(m->dir_nodes, dn.data(), m->n_dir * sizeof(int64_t), cudaMemcpyHostToDevice,
                                c->stream));
      SCVS_CUDA(cudaStreamSynchronize(c->stream));
    }
  } catch (...) {
    m->arena.release();
    delete m;
    throw;
  }
  c->meshes.push_back(m);
  return (int)c->meshes.size() - 1;
}

// |omega_k| rho and omega_k rho per mode, FP64 and FP32 (depend on rho)
void update_mode_scalars(Ctx &c, Mesh &m) {
  std::vector<double> wa(m.ld), wr(m.ld);
  std::vector<float> waf(m.ld), wrf(m.ld);
  for (int k = 0; k < m.ld; ++k) {
    wa[k] = std::fabs(m.omega[k]) * m.rho;
    wr[k] = m.omega[k] * m.rho;
    waf[k] = (float)wa[k];
    wrf[k] = (float)wr[k];
  }
  SCVS_CUDA(cudaMemcpyAsync(m.wabs_d, wa.data(), m.ld * sizeof(double), cudaMemcpyHostToDevice, c.stream));
  SCVS_CUDA(cudaMemcpyAsync(m.wrho_d, wr.data(), m.ld * sizeof(double), cudaMemcpyHostToDevice, c.stream));
  SCVS_CUDA(cudaMemcpyAsync(m.wabs_f, waf.data(), m.ld * sizeof(float), cudaMemcpyHostToDevice, c.stream));
  SCVS_CUDA(cudaMemcpyAsync(m.wrho_f, wrf.data(), m.ld * sizeof(float), cudaMemcpyHostToDevice, c.stream));
  SCVS_CUDA(cudaStreamSynchronize(c.stream));
}

int set_modes(scvs_ctx *c, int mesh_id, int n_modes, const double *omega, const void *g, bool on_device) {
  Mesh *m = get_mesh(c, mesh_id);
  if (!m) return fail(c, SCVS_ERR_ARG, "bad mesh id");
  if (n_modes < 1 || n_modes > 128) return fail(c, SCVS_ERR_ARG, "n_modes must be in [1, 128]");
  if (!omega || (!g && m->n_dir > 0)) return fail(c, SCVS_ERR_ARG, "null omega or g");
  m->mode_arena.release();
  m->neu = nullptr;
  m->pc = PcTables{};
  m->mpl_spmm = m->mpl_cheb = 0;
  m->tile_spmm = m->tile_cheb = 0;
  m->solved = false;
  m->m = n_modes;
  m->ld = mode_stride(n_modes);
  m->omega.assign(m->ld, 0.0);
  for (int k = 0; k < n_modes; ++k) m->omega[k] = omega[k];
  m->omega_d = m->mode_arena.alloc<double>(m->ld);
  SCVS_CUDA(cudaMemcpyAsync(m->omega_d, m->omega.data(), m->ld * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  m->wabs_d = m->mode_arena.alloc<double>(m->ld);
  m->wrho_d = m->mode_arena.alloc<double>(m->ld);
  m->wabs_f = m->mode_arena.alloc<float>(m->ld);
  m->wrho_f = m->mode_arena.alloc<float>(m->ld);
  update_mode_scalars(*c, *m);
  const int64_t gcount = (int64_t)n_modes * m->n_dir * m->dim;
  m->g = m->mode_arena.alloc<double2>(std::max<int64_t>(1, gcount));
  if (gcount)
    SCVS_CUDA(cudaMemcpyAsync(m->g, g, gcount * sizeof(double2), on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                              c->stream));
  const int64_t total = m->n_dof * m->ld;
  m->b = m->mode_arena.alloc<double2>(total);
  m->x = m->mode_arena.alloc<double2>(total);
  SCVS_CUDA(cudaMemsetAsync(m->x, 0, total * sizeof(double2), c->stream));
  lift_rhs(*c, *m);
  spectral_bounds(*c, *m);
  if (c->opts.autotune) {
    const std::vector<int64_t> key{m->dim, m->N, m->P, m->s_nnz, m->g_nnz, m->ld, m->n_comp};
    auto it = c->tune_cache.find(key);
    if (it == c->tune_cache.end()) {
      autotune_shapes(*c, *m);
      c->tune_cache[key] =
          Ctx::TuneRec{m->mpl_spmm, m->tile_spmm, m->mpl_cheb, m->tile_cheb, m->st_spmm, m->st_cheb, m->tune_us};
    } else {
      m->mpl_spmm = it->second.mpl_spmm;
      m->tile_spmm = it->second.tile_spmm;
      m->mpl_cheb = it->second.mpl_cheb;
      m->tile_cheb = it->second.tile_cheb;
      m->st_spmm = it->second.st_spmm;
      m->st_cheb = it->second.st_cheb;
      m->tune_us = it->second.us;
    }
  } else {
    m->st_spmm = m->st_cheb = c->opts.stage > 0 ? c->opts.stage : 0;
  }
  return SCVS_OK;
}

}  // namespace

extern "C" {

void scvs_default_opts(scvs_opts *o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->tol = 1e-8;
  o->restart = 30;
  o->precision = SCVS_PREC_MIXED;
  o->precond = SCVS_PC_AUTO;
  o->cheb_u = 2;
  o->cheb_c = 16;
  o->autotune = 1;
  o->cheb_m = 4;
  o->cheb_l = 75;
  o->max_cycles = 400;
  o->guess = SCVS_GUESS_ZERO;
  o->verbose = 0;
  o->stream = nullptr;
  o->schur_agg = 16;
  o->krylov = SCVS_KRYLOV_FGMRES;
  o->inner_max = 400;
  o->stage = -1;
  o->lap_size = 0;
  o->lap_smooth = 0;
}

// The option ranges documented in the header (scvs_create and scvs_set_opts).
static bool opts_valid(const scvs_opts *o) {
  return o->tol > 0 && o->restart >= 1 && o->restart <= 64 && o->cheb_u >= 1 && o->cheb_m >= 1 && o->cheb_l >= 1 &&
         o->cheb_c >= 1 && o->max_cycles >= 1 && o->precond >= 0 && o->precond <= SCVS_PC_AUTO &&
         o->schur_agg >= 0 && o->schur_agg <= 512 &&
         (o->stage == -1 || o->stage == 0 || o->stage == 4 || o->stage == 8 || o->stage == 16 || o->stage == 32) &&
         (o->krylov == SCVS_KRYLOV_FGMRES || o->krylov == SCVS_KRYLOV_COCR) && o->inner_max >= 1 &&
         o->lap_size >= -1 && o->lap_size <= 4096 && o->lap_smooth >= 0 && o->lap_smooth <= 64;
}

int scvs_create(scvs_ctx **out, const scvs_opts *opts) {
  if (!out) return SCVS_ERR_ARG;
  *out = nullptr;
  scvs_opts o;
  if (opts) o = *opts; else scvs_default_opts(&o);
  if (!opts_valid(&o)) return SCVS_ERR_ARG;
  scvs_ctx *c = new (std::nothrow) scvs_ctx();
  if (!c) return SCVS_ERR_OOM;
  c->opts = o;
  int r = guarded(c, [&]() {
    SCVS_CUDA(cudaGetDevice(&c->device));
    SCVS_CUDA(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device));
    c->stream = static_cast<cudaStream_t>(c->opts.stream);
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = c->device;
    SCVS_CUDA(cudaMemPoolCreate(&c->pool, &props));
    uint64_t keep = UINT64_MAX;  // never hand freed memory back: re-used by the next mesh / solve
    SCVS_CUDA(cudaMemPoolSetAttribute(c->pool, cudaMemPoolAttrReleaseThreshold, &keep));
    c->work.pool = c->pool;
    c->work.stream = c->stream;
    c->dev_err = c->work.alloc<int>(1);
    c->gsync = c->work.alloc<GridSync>(1);
    SCVS_CUDA(cudaMemset(c->dev_err, 0, sizeof(int)));
    SCVS_CUDA(cudaMemset(c->gsync, 0, sizeof(GridSync)));
    reference_tables(2, &c->ref2);
    reference_tables(3, &c->ref3);
    quad_tables(2, ISO_QUAD, &c->quad2);
    quad_tables(3, ISO_QUAD, &c->quad3);
    matfree_tables(*c);
    return SCVS_OK;
  });
  if (r != SCVS_OK) {
    c->work.release();
    if (c->pool) {
      if (c->stream) cudaStreamSynchronize(c->stream); else cudaDeviceSynchronize();
      cudaMemPoolDestroy(c->pool);
    }
    delete c;
    return r;
  }
  *out = c;
  return SCVS_OK;
}

void scvs_destroy(scvs_ctx *c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream); else cudaDeviceSynchronize();
  for (Mesh *m : c->meshes) {
    if (!m) continue;
    m->mode_arena.release();
    m->arena.release();
    delete m;
  }
  c->timers.destroy();
  c->guess.release();
  c->work.release();
  if (c->pool) {
    if (c->stream) cudaStreamSynchronize(c->stream); else cudaDeviceSynchronize();
    cudaMemPoolDestroy(c->pool);
  }
  delete c;
}

const char *scvs_last_error(const scvs_ctx *c) { return c ? c->err.c_str() : "null context"; }

int scvs_set_opts(scvs_ctx *c, const scvs_opts *o) {
  if (!c || !o) return SCVS_ERR_ARG;
  if (!opts_valid(o)) return fail(c, SCVS_ERR_ARG, "invalid options");
  void *old_stream = c->opts.stream;
  if (o->stream != old_stream) {
    // work queued on the old stream finishes before the arenas follow the new one
    if (c->stream) cudaStreamSynchronize(c->stream); else cudaDeviceSynchronize();
    c->stream = static_cast<cudaStream_t>(o->stream);
    c->work.stream = c->stream;
    for (Mesh *m : c->meshes)
      if (m) { m->arena.stream = c->stream; m->mode_arena.stream = c->stream; }
  }
  c->opts = *o;
  return SCVS_OK;
}

int scvs_set_mesh(scvs_ctx *c, int32_t dim, int64_t N, int64_t P, const double *xyz, int64_t E, const int32_t *conn,
                  const uint8_t *tag) {
  return guarded(c, [&]() { return add_mesh(c, dim, N, P, xyz, E, conn, tag, false); });
}

int scvs_set_mesh_dev(scvs_ctx *c, int32_t dim, int64_t N, int64_t P, const double *xyz, int64_t E,
                      const int32_t *conn, const uint8_t *tag) {
  return guarded(c, [&]() { return add_mesh(c, dim, N, P, xyz, E, conn, tag, true); });
}

int scvs_clear_meshes(scvs_ctx *c) {
  return guarded(c, [&]() {
    SCVS_CUDA(cudaStreamSynchronize(c->stream));
    for (Mesh *m : c->meshes) {
      if (!m) continue;
      m->mode_arena.release();
      m->arena.release();
      delete m;
    }
    c->meshes.clear();
    return SCVS_OK;
  });
}

int scvs_set_components(scvs_ctx *c, int32_t mesh_id, int32_t n_comp, const int32_t *node_comp) {
  return guarded(c, [&]() {
    Mesh *m = get_mesh(c, mesh_id);
    if (!m) return fail(c, SCVS_ERR_ARG, "bad mesh id");
    if (n_comp < 1 || n_comp > 65536 || (n_comp > 1 && !node_comp))
      return fail(c, SCVS_ERR_ARG, "n_comp must be in [1, 65536] with a node_comp array");
    if (node_comp)
      for (int64_t i = 0; i < m->N; ++i)
        if (node_comp[i] < 0 || node_comp[i] >= n_comp) return fail(c, SCVS_ERR_ARG, "node_comp out of range");
    // no matrix entry may couple two components
    if (node_comp && n_comp > 1) {
      std::vector<int64_t> sp(m->N + 1);
      std::vector<int32_t> sc(m->s_nnz);
      SCVS_CUDA(cudaMemcpy(sp.data(), m->s_ptr, sp.size() * sizeof(int64_t), cudaMemcpyDeviceToHost));
      SCVS_CUDA(cudaMemcpy(sc.data(), m->s_col, sc.size() * sizeof(int32_t), cudaMemcpyDeviceToHost));
      for (int64_t r = 0; r < m->N; ++r)
        for (int64_t t = sp[r]; t < sp[r + 1]; ++t)
          if (node_comp[sc[t]] != node_comp[r]) return fail(c, SCVS_ERR_MESH, "an element spans two components");
    }
    set_chunks(*c, *m, n_comp > 1 ? node_comp : nullptr, n_comp);
    if (m->m > 0) {  // modes already set: per-system norms of the right-hand sides
      lift_rhs(*c, *m);
      m->solved = false;
    }
    return SCVS_OK;
  });
}

int scvs_set_physics(scvs_ctx *c, int32_t mesh_id, double rho, double mu) {
  return guarded(c, [&]() {
    Mesh *m = get_mesh(c, mesh_id);
    if (!m) return fail(c, SCVS_ERR_ARG, "bad mesh id");
    if (!(rho > 0) || !(mu > 0)) return fail(c, SCVS_ERR_ARG, "rho and mu must be positive");
    m->rho = rho;
    m->mu = mu;
    if (m->m > 0) {  // modes already set: rebuild what depends on rho, mu
      update_mode_scalars(*c, *m);
      m->pc = PcTables{};
      m->solved = false;
      lift_rhs(*c, *m);
      spectral_bounds(*c, *m);
    }
    return SCVS_OK;
  });
}

int scvs_dirichlet_count(scvs_ctx *c, int32_t mesh_id, int64_t *n) {
  return guarded(c, [&]() {
    Mesh *m = get_mesh(c, mesh_id);
    if (!m || !n) return fail(c, SCVS_ERR_ARG, "bad argument");
    *n = m->n_dir;
    return SCVS_OK;
  });
}

int scvs_set_modes(scvs_ctx *c, int32_t mesh_id, int32_t n_modes, const double *omega, const scvs_c64 *g) {
  return guarded(c, [&]() { return set_modes(c, mesh_id, n_modes, omega, g, false); });
}

int scvs_set_modes_dev(scvs_ctx *c, int32_t mesh_id, int32_t n_modes, const double *omega, const void *g) {
  return guarded(c, [&]() { return set_modes(c, mesh_id, n_modes, omega, g, true); });
}

int scvs_solve(scvs_ctx *c, int32_t mesh_id, scvs_mode_report *rep, int64_t rep_len) {
  return guarded(c, [&]() {
    std::vector<Mesh *> todo;
    if (mesh_id < 0) {
      for (Mesh *m : c->meshes) if (m) todo.push_back(m);
    } else {
      Mesh *m = get_mesh(c, mesh_id);
      if (!m) return fail(c, SCVS_ERR_ARG, "bad mesh id");
      todo.push_back(m);
    }
    for (Mesh *m : todo)
      if (m->m == 0) return fail(c, SCVS_ERR_STATE, "scvs_set_modes must precede scvs_solve");
    int64_t pos = 0;
    for (Mesh *m : todo) {
      int r = solve_mesh(*c, *m);
      if (r != SCVS_OK) return fail(c, r, r == SCVS_ERR_TIMEOUT ? "a device grid barrier timed out" : "solve failed");
      m->solved = true;
      for (size_t k = 0; k < m->rep.size(); ++k, ++pos)
        if (rep && pos < rep_len) rep[pos] = m->rep[k];
    }
    return SCVS_OK;
  });
}

int scvs_get_modal(scvs_ctx *c, int32_t mesh_id, scvs_c64 *u, scvs_c64 *p) {
  return guarded(c, [&]() {
    Mesh *m = get_mesh(c, mesh_id);
    if (!m || m->m == 0) return fail(c, SCVS_ERR_ARG, "bad mesh id or no modes");
    // transpose on the device into the caller's mode-major layout, then one
    // copy per field straight into the caller's arrays (DMA when they are pinned)
    const int64_t nu = (int64_t)m->dim * m->N, np = m->P;
    double2 *U = nullptr, *Pm = nullptr;
    SCVS_CUDA(ctx_malloc(*c, &U, (size_t)m->m * nu * sizeof(double2), c->stream));
    SCVS_CUDA(ctx_malloc(*c, &Pm, (size_t)m->m * np * sizeof(double2), c->stream));
    modal_split(*c, *m, U, Pm);
    if (u) SCVS_CUDA(cudaMemcpyAsync(u, U, (size_t)m->m * nu * sizeof(double2), cudaMemcpyDeviceToHost, c->stream));
    if (p) SCVS_CUDA(cudaMemcpyAsync(p, Pm, (size_t)m->m * np * sizeof(double2), cudaMemcpyDeviceToHost, c->stream));
    SCVS_CUDA(cudaFreeAsync(U, c->stream));
    SCVS_CUDA(cudaFreeAsync(Pm, c->stream));
    SCVS_CUDA(cudaStreamSynchronize(c->stream));
    return SCVS_OK;
  });
}

int scvs_set_solution(scvs_ctx *c, int32_t mesh_id, const scvs_c64 *u, const scvs_c64 *p) {
  return guarded(c, [&]() {
    Mesh *m = get_mesh(c, mesh_id);
    if (!m || !u || !p) return fail(c, SCVS_ERR_ARG, "bad mesh id or null u / p");
    if (m->m == 0) return fail(c, SCVS_ERR_STATE, "call scvs_set_modes first");
    std::vector<double2> h((size_t)m->n_dof * m->ld, make_double2(0.0, 0.0));
    const int64_t nu = (int64_t)m->dim * m->N;
    for (int k = 0; k < m->m; ++k) {
      for (int64_t d = 0; d < nu; ++d) {
        const scvs_c64 v = u[(size_t)k * nu + d];
        h[(size_t)d * m->ld + k] = make_double2(v.re, v.im);
      }
      for (int64_t v = 0; v < m->P; ++v) {
        const scvs_c64 z = p[(size_t)k * m->P + v];
        h[(size_t)(nu + v) * m->ld + k] = make_double2(z.re, z.im);
      }
    }
    SCVS_CUDA(cudaMemcpyAsync(m->x, h.data(), h.size() * sizeof(double2), cudaMemcpyHostToDevice, c->stream));
    SCVS_CUDA(cudaStreamSynchronize(c->stream));
    m->solved = false;
    return SCVS_OK;
  });
}

int scvs_modal_dev(scvs_ctx *c, int32_t mesh_id, const void **x, int64_t *n_dof, int32_t *ld) {
  return guarded(c, [&]() {
    Mesh *m = get_mesh(c, mesh_id);
    if (!m || m->m == 0) return fail(c, SCVS_ERR_ARG, "bad mesh id or no modes");
    if (x) *x = m->x;
    if (n_dof) *n_dof = m->n_dof;
    if (ld) *ld = m->ld;
    return SCVS_OK;
  });
}

int scvs_reconstruct_dev(scvs_ctx *c, int32_t mesh_id, int32_t n_t, double period, double *u_t, double *p_t) {
  return guarded(c, [&]() {
    Mesh *m = get_mesh(c, mesh_id);
    if (!m || m->m == 0) return fail(c, SCVS_ERR_ARG, "bad mesh id or no modes");
    if (n_t < 1 || !(period > 0)) return fail(c, SCVS_ERR_ARG, "n_t >= 1 and period > 0 required");
    reconstruct(*c, *m, n_t, period, u_t, p_t);
    return SCVS_OK;
  });
}

int scvs_reconstruct_dev_static(scvs_ctx *c, int32_t mesh_id, int32_t n_t, double period, double *u_t, double *p_t) {
  return guarded(c, [&]() {
    Mesh *m = get_mesh(c, mesh_id);
    if (!m || m->m == 0) return fail(c, SCVS_ERR_ARG, "bad mesh id or no modes");
    if (n_t < 1 || !(period > 0)) return fail(c, SCVS_ERR_ARG, "n_t >= 1 and period > 0 required");
    if ((int64_t)n_t * m->m > SCVS_RECON_STATIC_MAX)
      return fail(c, SCVS_ERR_ARG, "n_t * n_modes exceeds SCVS_RECON_STATIC_MAX (" +
                                       std::to_string(SCVS_RECON_STATIC_MAX) + ") twiddles of the static table");
    reconstruct_static(*c, *m, n_t, period, u_t, p_t);
    return SCVS_OK;
  });
}

int scvs_reconstruct(scvs_ctx *c, int32_t mesh_id, int32_t n_t, double period, double *u_t, double *p_t) {
  return guarded(c, [&]() {
    Mesh *m = get_mesh(c, mesh_id);
    if (!m || m->m == 0) return fail(c, SCVS_ERR_ARG, "bad mesh id or no modes");
    if (n_t < 1 || !(period > 0)) return fail(c, SCVS_ERR_ARG, "n_t >= 1 and period > 0 required");
    const int64_t nu = (int64_t)n_t * m->dim * m->N, np = (int64_t)n_t * m->P;
    double *du = nullptr, *dp = nullptr;
    if (u_t) SCVS_CUDA(ctx_malloc(*c, &du, nu * sizeof(double), c->stream));
    if (p_t) SCVS_CUDA(ctx_malloc(*c, &dp, np * sizeof(double), c->stream));
    reconstruct(*c, *m, n_t, period, du, dp);
    if (u_t) SCVS_CUDA(cudaMemcpyAsync(u_t, du, nu * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    if (p_t) SCVS_CUDA(cudaMemcpyAsync(p_t, dp, np * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    if (du) SCVS_CUDA(cudaFreeAsync(du, c->stream));
    if (dp) SCVS_CUDA(cudaFreeAsync(dp, c->stream));
    SCVS_CUDA(cudaStreamSynchronize(c->stream));
    return SCVS_OK;
  });
}

int scvs_csr_size(scvs_ctx *c, int32_t mesh_id, int32_t which, int64_t *n_rows, int64_t *nnz) {
  return guarded(c, [&]() {
    Mesh *m = get_mesh(c, mesh_id);
    if (!m) return fail(c, SCVS_ERR_ARG, "bad mesh id");
    int64_t r, z;
    switch (which) {
      case SCVS_CSR_S: r = m->N; z = m->s_nnz; break;
      case SCVS_CSR_G: r = m->N; z = m->g_nnz; break;
      case SCVS_CSR_GT: r = m->P; z = m->gt_nnz; break;
      case SCVS_CSR_Q: r = m->P; z = m->q_nnz; break;
      default: return fail(c, SCVS_ERR_ARG, "bad pattern id");
    }
    if (n_rows) *n_rows = r;
    if (nnz) *nnz = z;
    return SCVS_OK;
  });
}

int scvs_get_csr(scvs_ctx *c, int32_t mesh_id, int32_t which, int64_t *rowptr, int32_t *col) {
  return guarded(c, [&]() {
    Mesh *m = get_mesh(c, mesh_id);
    if (!m || !rowptr || !col) return fail(c, SCVS_ERR_ARG, "bad argument");
    std::vector<int64_t> sp(m->N + 1), gp(m->N + 1);
    std::vector<int32_t> sc(m->s_nnz);
    SCVS_CUDA(cudaMemcpy(sp.data(), m->s_ptr, sp.size() * sizeof(int64_t), cudaMemcpyDeviceToHost));
    SCVS_CUDA(cudaMemcpy(gp.data(), m->g_ptr, gp.size() * sizeof(int64_t), cudaMemcpyDeviceToHost));
    SCVS_CUDA(cudaMemcpy(sc.data(), m->s_col, sc.size() * sizeof(int32_t), cudaMemcpyDeviceToHost));
    // S rows hold, in this order, the G part (columns < P) and the rest
    auto emit = [&](int64_t rows, bool g_part) {
      int64_t pos = 0;
      for (int64_t r = 0; r < rows; ++r) {
        rowptr[r] = pos;
        int64_t len = g_part ? gp[r + 1] - gp[r] : sp[r + 1] - sp[r];
        std::memcpy(col + pos, sc.data() + sp[r], len * sizeof(int32_t));
        pos += len;
      }
      rowptr[rows] = pos;
    };
    switch (which) {
      case SCVS_CSR_S: emit(m->N, false); break;
      case SCVS_CSR_G: emit(m->N, true); break;
      case SCVS_CSR_GT: emit(m->P, false); break;
      case SCVS_CSR_Q: emit(m->P, true); break;
      default: return fail(c, SCVS_ERR_ARG, "bad pattern id");
    }
    return SCVS_OK;
  });
}

int scvs_get_values(scvs_ctx *c, int32_t mesh_id, int32_t which, double *vals) {
  return guarded(c, [&]() {
    Mesh *m = get_mesh(c, mesh_id);
    if (!m || !vals) return fail(c, SCVS_ERR_ARG, "bad argument");
    auto cp = [&](double *dst, const double *src, int64_t n) {
      SCVS_CUDA(cudaMemcpy(dst, src, n * sizeof(double), cudaMemcpyDeviceToHost));
    };
    switch (which) {
      case SCVS_CSR_S: cp(vals, m->Ms, m->s_nnz); cp(vals + m->s_nnz, m->Ks, m->s_nnz); break;
      case SCVS_CSR_G: cp(vals, m->Dv, (int64_t)m->dim * m->g_nnz); break;
      case SCVS_CSR_GT: cp(vals, m->DTv, (int64_t)m->dim * m->gt_nnz); break;
      case SCVS_CSR_Q: cp(vals, m->Mp, m->q_nnz); cp(vals + m->q_nnz, m->Lp, m->q_nnz); break;
      default: return fail(c, SCVS_ERR_ARG, "bad pattern id");
    }
    return SCVS_OK;
  });
}

int scvs_mode_stride(scvs_ctx *c, int32_t mesh_id, int32_t *ld) {
  return guarded(c, [&]() {
    Mesh *m = get_mesh(c, mesh_id);
    if (!m || !ld || m->m == 0) return fail(c, SCVS_ERR_ARG, "bad mesh id or no modes");
    *ld = m->ld;
    return SCVS_OK;
  });
}

int scvs_dof_count(scvs_ctx *c, int32_t mesh_id, int64_t *n) {
  return guarded(c, [&]() {
    Mesh *m = get_mesh(c, mesh_id);
    if (!m || !n) return fail(c, SCVS_ERR_ARG, "bad argument");
    *n = m->n_dof;
    return SCVS_OK;
  });
}

int scvs_apply(scvs_ctx *c, int32_t mesh_id, int32_t precision, const void *x, void *y) {
  return guarded(c, [&]() {
    Mesh *m = get_mesh(c, mesh_id);
    if (!m || m->m == 0 || !x || !y) return fail(c, SCVS_ERR_ARG, "bad argument");
    if (precision == SCVS_PREC_FP64)
      apply_saddle<double>(*c, *m, static_cast<const double2 *>(x), static_cast<double2 *>(y));
    else if (precision == SCVS_PREC_MIXED)
      apply_saddle<float>(*c, *m, static_cast<const float2 *>(x), static_cast<float2 *>(y));
    else
      return fail(c, SCVS_ERR_ARG, "bad precision");
    SCVS_CUDA(cudaGetLastError());
    return SCVS_OK;
  });
}

int scvs_apply_matfree(scvs_ctx *c, int32_t mesh_id, int32_t precision, const void *x, void *y) {
  return guarded(c, [&]() {
    Mesh *m = get_mesh(c, mesh_id);
    if (!m || m->m == 0 || !x || !y) return fail(c, SCVS_ERR_ARG, "bad argument");
    if (precision != SCVS_PREC_FP64 && precision != SCVS_PREC_MIXED) return fail(c, SCVS_ERR_ARG, "bad precision");
    apply_matfree(*c, *m, precision, x, y);
    SCVS_CUDA(cudaGetLastError());
    return SCVS_OK;
  });
}

int scvs_rhs_dev(scvs_ctx *c, int32_t mesh_id, const void **b) {
  return guarded(c, [&]() {
    Mesh *m = get_mesh(c, mesh_id);
    if (!m || m->m == 0 || !b) return fail(c, SCVS_ERR_ARG, "bad argument");
    *b = m->b;
    return SCVS_OK;
  });
}

int scvs_apply_precond(scvs_ctx *c, int32_t mesh_id, const void *r, void *z) {
  return guarded(c, [&]() {
    Mesh *m = get_mesh(c, mesh_id);
    if (!m || !r || !z) return fail(c, SCVS_ERR_ARG, "bad argument");
    if (m->m == 0) return fail(c, SCVS_ERR_STATE, "scvs_set_modes has not been called for this mesh");
    float2 *s = nullptr;
    SCVS_CUDA(ctx_malloc(*c, &s, precond_scratch_elems(*m) * sizeof(float2), c->stream));
    apply_precond<float>(*c, *m, static_cast<const float2 *>(r), static_cast<float2 *>(z), s, nullptr);
    SCVS_CUDA(cudaFreeAsync(s, c->stream));
    SCVS_CUDA(cudaGetLastError());
    // the persistent pressure and coarse solves wait at bounded grid barriers
    int gerr = 0;
    SCVS_CUDA(cudaMemcpyAsync(&gerr, &c->gsync->err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    SCVS_CUDA(cudaStreamSynchronize(c->stream));
    if (gerr) {
      SCVS_CUDA(cudaMemsetAsync(c->gsync, 0, sizeof(GridSync), c->stream));
      SCVS_CUDA(cudaStreamSynchronize(c->stream));
      return fail(c, SCVS_ERR_TIMEOUT, "a grid barrier of the preconditioner gave up; z is void");
    }
    return SCVS_OK;
  });
}

int64_t scvs_launch_count(const scvs_ctx *c) { return c ? c->launches.n : -1; }

int scvs_pool_usage(scvs_ctx *c, int32_t reset_high, int64_t *used, int64_t *used_high, int64_t *reserved) {
  return guarded(c, [&]() {
    SCVS_CUDA(cudaStreamSynchronize(c->stream));
    unsigned long long u = 0, h = 0, r = 0;  // the runtime reports these attributes as 64-bit counts
    SCVS_CUDA(cudaMemPoolGetAttribute(c->pool, cudaMemPoolAttrUsedMemCurrent, &u));
    SCVS_CUDA(cudaMemPoolGetAttribute(c->pool, cudaMemPoolAttrUsedMemHigh, &h));
    SCVS_CUDA(cudaMemPoolGetAttribute(c->pool, cudaMemPoolAttrReservedMemCurrent, &r));
    if (used) *used = (int64_t)u;
    if (used_high) *used_high = (int64_t)h;
    if (reserved) *reserved = (int64_t)r;
    if (reset_high) {
      unsigned long long z = 0;
      SCVS_CUDA(cudaMemPoolSetAttribute(c->pool, cudaMemPoolAttrUsedMemHigh, &z));
    }
    return SCVS_OK;
  });
}

void scvs_default_train_opts(scvs_train_opts *o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->n_pod = 32;
  o->hidden = 256;
  o->steps = 3000;
  o->batch = 256;
  o->lr = 1e-3;
  o->seed = 0;
  o->max_pod_snapshots = 512;
}

int scvs_guess_add_snapshots(scvs_ctx *c, int32_t mesh_id, const double *features) {
  return guarded(c, [&]() {
    Mesh *m = get_mesh(c, mesh_id);
    if (!m || !features) return fail(c, SCVS_ERR_ARG, "bad argument");
    if (!m->solved) return fail(c, SCVS_ERR_STATE, "solve the mesh before adding its modes as snapshots");
    guess_add_snapshots(*c, *m, features);
    return SCVS_OK;
  });
}

int scvs_train_guess(scvs_ctx *c, const scvs_train_opts *o, double *loss) {
  return guarded(c, [&]() {
    scvs_train_opts d;
    scvs_default_train_opts(&d);
    const scvs_train_opts &oo = o ? *o : d;
    if (oo.n_pod < 1 || oo.hidden < 1 || oo.hidden > 1024 || oo.steps < 0 || oo.batch < 1 || !(oo.lr > 0) ||
        oo.max_pod_snapshots < 2)
      return fail(c, SCVS_ERR_ARG, "invalid training options");
    if (c->guess.n_snap < 4) return fail(c, SCVS_ERR_STATE, "fewer than 4 snapshots");
    const double l = guess_train(*c, oo);
    if (loss) *loss = l;
    return SCVS_OK;
  });
}

int scvs_guess_set_features(scvs_ctx *c, int32_t mesh_id, const double *features) {
  return guarded(c, [&]() {
    Mesh *m = get_mesh(c, mesh_id);
    if (!m || !features || m->m == 0) return fail(c, SCVS_ERR_ARG, "bad mesh id, features, or no modes");
    m->feat.assign(features, features + 5 * m->m);
    return SCVS_OK;
  });
}

int scvs_guess_info(scvs_ctx *c, int64_t *n_snap, int32_t *n_pod, int32_t *trained) {
  return guarded(c, [&]() {
    if (n_snap) *n_snap = c->guess.n_snap;
    if (n_pod) *n_pod = c->guess.n_pod;
    if (trained) *trained = c->guess.trained ? 1 : 0;
    return SCVS_OK;
  });
}

int scvs_guess_reset(scvs_ctx *c) {
  return guarded(c, [&]() {
    SCVS_CUDA(cudaStreamSynchronize(c->stream));
    c->guess.release();
    return SCVS_OK;
  });
}

int scvs_mlp_init(scvs_ctx *c, int32_t n_in, int32_t hidden, int32_t n_out, const float *params) {
  return guarded(c, [&]() {
    if (n_in < 1 || hidden < 1 || hidden > 1024 || n_out < 1 || !params) return fail(c, SCVS_ERR_ARG, "bad MLP sizes");
    GuessModel &g = c->guess;
    mlp_alloc(g, n_in, hidden, n_out);
    SCVS_CUDA(cudaMemcpy(g.Wf, params, g.n_params * sizeof(float), cudaMemcpyHostToDevice));
    mlp_refresh_bf16(*c, g);
    SCVS_CUDA(cudaStreamSynchronize(c->stream));
    return SCVS_OK;
  });
}

int scvs_mlp_set_params(scvs_ctx *c, const float *params) {
  return guarded(c, [&]() {
    GuessModel &g = c->guess;
    if (!params) return fail(c, SCVS_ERR_ARG, "null parameters");
    if (g.n_params == 0) return fail(c, SCVS_ERR_STATE, "no MLP (scvs_mlp_init or scvs_train_guess first)");
    SCVS_CUDA(cudaMemcpy(g.Wf, params, g.n_params * sizeof(float), cudaMemcpyHostToDevice));
    mlp_refresh_bf16(*c, g);
    SCVS_CUDA(cudaStreamSynchronize(c->stream));
    return SCVS_OK;
  });
}

int scvs_guess_basis(scvs_ctx *c, int32_t block, int64_t n_rows, int32_t n_pod, scvs_c64 *phi) {
  return guarded(c, [&]() {
    GuessModel &g = c->guess;
    if (!g.trained || !g.Phi_u) return fail(c, SCVS_ERR_STATE, "no trained guess");
    if (block != 0 && block != 1) return fail(c, SCVS_ERR_ARG, "block must be 0 (velocity) or 1 (pressure)");
    const int64_t nr = block == 0 ? g.n_u : g.n_dof - g.n_u;
    if (!phi || n_rows != nr || n_pod != g.n_pod) return fail(c, SCVS_ERR_ARG, "basis size mismatch");
    std::vector<float2> h((size_t)nr * g.n_pod);
    SCVS_CUDA(cudaMemcpy(h.data(), block == 0 ? g.Phi_u : g.Phi_p, h.size() * sizeof(float2), cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < h.size(); ++i) phi[i] = scvs_c64{h[i].x, h[i].y};
    return SCVS_OK;
  });
}

int scvs_guess_coefficients(scvs_ctx *c, int32_t block, int64_t n_snap, int32_t n_pod, scvs_c64 *a) {
  return guarded(c, [&]() {
    GuessModel &g = c->guess;
    if (!g.trained || g.coef_u.empty()) return fail(c, SCVS_ERR_STATE, "no trained guess");
    if (block != 0 && block != 1) return fail(c, SCVS_ERR_ARG, "block must be 0 (velocity) or 1 (pressure)");
    if (!a || n_snap != g.n_snap || n_pod != g.n_pod) return fail(c, SCVS_ERR_ARG, "coefficient size mismatch");
    const auto &src = block == 0 ? g.coef_u : g.coef_p;
    for (size_t i = 0; i < src.size(); ++i) a[i] = scvs_c64{src[i].real(), src[i].imag()};
    return SCVS_OK;
  });
}

int scvs_guess_initial(scvs_ctx *c, int32_t mesh_id, int64_t n_modes, double *res0, int32_t *kept) {
  return guarded(c, [&]() {
    Mesh *m = get_mesh(c, mesh_id);
    if (!m || m->m == 0) return fail(c, SCVS_ERR_ARG, "bad mesh id or no modes");
    if (!res0 || !kept || n_modes != m->m) return fail(c, SCVS_ERR_ARG, "res0/kept must hold one entry per mode");
    std::vector<int> k(m->m, 0);
    if (!guess_probe(*c, *m, res0, k.data()))
      return fail(c, SCVS_ERR_STATE,
                  "the learned guess cannot serve this mesh (untrained model, another node set, no features, or "
                  "several components)");
    for (int i = 0; i < m->m; ++i) kept[i] = k[i];
    return SCVS_OK;
  });
}

int scvs_mlp_num_params(scvs_ctx *c, int64_t *n) {
  return guarded(c, [&]() {
    if (!n) return fail(c, SCVS_ERR_ARG, "null");
    *n = c->guess.n_params;
    return SCVS_OK;
  });
}

int scvs_mlp_get_params(scvs_ctx *c, float *params) {
  return guarded(c, [&]() {
    if (!params || c->guess.n_params == 0) return fail(c, SCVS_ERR_STATE, "no MLP");
    SCVS_CUDA(cudaMemcpy(params, c->guess.Wf, c->guess.n_params * sizeof(float), cudaMemcpyDeviceToHost));
    return SCVS_OK;
  });
}

int scvs_mlp_forward_dev(scvs_ctx *c, const float *x, int64_t B, float *y) {
  return guarded(c, [&]() {
    if (!x || !y || B < 1 || c->guess.n_params == 0) return fail(c, SCVS_ERR_ARG, "bad argument or no MLP");
    mlp_forward(*c, c->guess, x, B, y);
    SCVS_CUDA(cudaGetLastError());
    return SCVS_OK;
  });
}

int scvs_mlp_gradient_dev(scvs_ctx *c, const float *x, const float *t, int64_t B, float *grad, double *loss) {
  return guarded(c, [&]() {
    if (!x || !t || B < 1 || c->guess.n_params == 0) return fail(c, SCVS_ERR_ARG, "bad argument or no MLP");
    const float l = mlp_gradient(*c, c->guess, x, t, B);
    if (grad)
      SCVS_CUDA(cudaMemcpy(grad, c->guess.grad, c->guess.n_params * sizeof(float), cudaMemcpyDeviceToHost));
    if (loss) *loss = l;
    return SCVS_OK;
  });
}

int scvs_mlp_adam_step(scvs_ctx *c, double lr) {
  return guarded(c, [&]() {
    if (c->guess.n_params == 0 || !(lr > 0)) return fail(c, SCVS_ERR_ARG, "no MLP or bad lr");
    mlp_adam(*c, c->guess, (float)lr);
    SCVS_CUDA(cudaStreamSynchronize(c->stream));
    return SCVS_OK;
  });
}

int scvs_tuned_shapes(scvs_ctx *c, int32_t mesh_id, int32_t *shape, float *us) {
  return guarded(c, [&]() {
    Mesh *m = get_mesh(c, mesh_id);
    if (!m) return fail(c, SCVS_ERR_ARG, "bad mesh id");
    if (shape) {
      shape[0] = m->mpl_spmm;
      shape[1] = m->tile_spmm;
      shape[2] = m->mpl_cheb;
      shape[3] = m->tile_cheb;
    }
    if (us)
      for (int i = 0; i < 2 * 3 * SCVS_TUNE_TILES; ++i) us[i] = i < (int)m->tune_us.size() ? m->tune_us[i] : 0.0f;
    return SCVS_OK;
  });
}

int scvs_staged_info(scvs_ctx *c, int32_t mesh_id, int64_t *info, float *us) {
  return guarded(c, [&]() {
    Mesh *m = get_mesh(c, mesh_id);
    if (!m) return fail(c, SCVS_ERR_ARG, "bad mesh id");
    const RowBlocks &rb = m->rb;
    if (info) {
      const void *aligned = reinterpret_cast<const void *>(256);  // any 16-byte aligned vector
      const int64_t v[10] = {rb.valid ? 1 : 0, rb.n_blk, rb.budget, rb.fp_max, rb.fv_max, rb.fp_total, m->st_spmm,
                             m->st_cheb, staged_ok(*c, *m, m->st_spmm, true, aligned) ? 1 : 0,
                             staged_ok(*c, *m, m->st_cheb, false, aligned) ? 1 : 0};
      for (int i = 0; i < 10; ++i) info[i] = v[i];
    }
    if (us) {
      const size_t st0 = (size_t)2 * 3 * SCVS_TUNE_TILES;
      for (int i = 0; i < 8; ++i) us[i] = st0 + i < m->tune_us.size() ? m->tune_us[st0 + i] : 0.0f;
    }
    return SCVS_OK;
  });
}

int scvs_staged_blocks(scvs_ctx *c, int32_t mesh_id, int32_t *perm, int64_t *row0, int64_t *fp_ptr, int32_t *fp_col,
                       int32_t *fv_len, uint16_t *lcol) {
  return guarded(c, [&]() {
    Mesh *m = get_mesh(c, mesh_id);
    if (!m) return fail(c, SCVS_ERR_ARG, "bad mesh id");
    const RowBlocks &rb = m->rb;
    if (!rb.valid) return fail(c, SCVS_ERR_STATE, "the mesh has no row blocks");
    auto cp = [&](void *dst, const void *src, size_t bytes) {
      if (dst) SCVS_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, c->stream));
    };
    cp(perm, rb.perm, m->N * sizeof(int32_t));
    cp(row0, rb.row0, (rb.n_blk + 1) * sizeof(int64_t));
    cp(fp_ptr, rb.fp_ptr, (rb.n_blk + 1) * sizeof(int64_t));
    cp(fp_col, rb.fp_col, rb.fp_total * sizeof(int32_t));
    cp(fv_len, rb.fv_len, rb.n_blk * sizeof(int32_t));
    cp(lcol, rb.lcol, m->s_nnz * sizeof(uint16_t));
    SCVS_CUDA(cudaStreamSynchronize(c->stream));
    return SCVS_OK;
  });
}

int scvs_set_neumann(scvs_ctx *c, int32_t mesh_id, const scvs_c64 *h, int64_t *n_faces) {
  return guarded(c, [&]() {
    Mesh *m = get_mesh(c, mesh_id);
    if (!m || !h) return fail(c, SCVS_ERR_ARG, "bad mesh id or null h");
    if (m->m == 0) return fail(c, SCVS_ERR_STATE, "call scvs_set_modes first");
    const int64_t nf = set_neumann(*c, *m, reinterpret_cast<const double2 *>(h));
    m->solved = false;
    lift_rhs(*c, *m);
    if (n_faces) *n_faces = nf;
    return SCVS_OK;
  });
}

int scvs_bc_spectrum(scvs_ctx *c, int32_t n_t, int64_t n_pts, int32_t n_modes, const double *g_t, const double *w,
                     void *c_out, double *e2) {
  return guarded(c, [&]() {
    if (n_t < 2 || n_pts < 1 || n_modes < 1 || 2 * (int64_t)(n_modes - 1) >= n_t)
      return fail(c, SCVS_ERR_ARG, "need n_t >= 2, n_pts >= 1, 1 <= n_modes and 2 (n_modes - 1) < n_t");
    if ((int64_t)n_t * n_pts > (int64_t)1 << 40 || (int64_t)n_modes * n_pts > (int64_t)1 << 40)
      return fail(c, SCVS_ERR_ARG, "sizes too large");
    if (!g_t || !c_out || !e2) return fail(c, SCVS_ERR_ARG, "null g_t, c or e2");
    bc_spectrum(*c, n_t, n_pts, n_modes, g_t, w, static_cast<double2 *>(c_out), e2);
    return SCVS_OK;
  });
}

int scvs_mode_energies(scvs_ctx *c, int32_t mesh_id, int64_t n_out, double *E, double *incr2) {
  return guarded(c, [&]() {
    Mesh *m = get_mesh(c, mesh_id);
    if (!m) return fail(c, SCVS_ERR_ARG, "bad mesh id");
    if (!m->solved) return fail(c, SCVS_ERR_STATE, "no solution: call scvs_solve first");
    if (!E || n_out < (int64_t)m->n_comp * m->m)
      return fail(c, SCVS_ERR_ARG, "E needs n_components * n_modes entries");
    mode_energies(*c, *m, E, incr2);
    return SCVS_OK;
  });
}

// ---- checkpoint files (host only) -----------------------------------------
// FNV-1a 64-bit hash (Fowler, Noll, Vo): h = (h xor byte) * 1099511628211 from
// 14695981039346656037.
static uint64_t fnv1a(uint64_t h, const void *data, size_t n) {
  const unsigned char *b = static_cast<const unsigned char *>(data);
  for (size_t i = 0; i < n; ++i) {
    h ^= b[i];
    h *= 1099511628211ULL;
  }
  return h;
}
static const uint64_t FNV_OFFSET = 14695981039346656037ULL;
static const char CKPT_MAGIC[8] = {'S', 'C', 'V', 'S', 'C', 'K', 'P', '2'};

int scvs_barrier_selftest(scvs_ctx *c, int64_t spin_limit, int32_t n_blocks, int32_t absent_block,
                          int32_t *blocks_passed) {
  return guarded(c, [&]() {
    if (spin_limit < 1 || spin_limit > SPIN_LIMIT || n_blocks < 1 || n_blocks > c->num_sms ||
        absent_block < -1 || absent_block >= n_blocks)
      return fail(c, SCVS_ERR_ARG, "spin_limit in [1, 2^24], 1 <= n_blocks <= SMs, -1 <= absent_block < n_blocks");
    int passed = 0;
    const int r = barrier_selftest(*c, (long long)spin_limit, n_blocks, absent_block, &passed);
    if (blocks_passed) *blocks_passed = passed;
    if (r == SCVS_ERR_TIMEOUT) return fail(c, r, "a device grid barrier timed out (self-test)");
    return r;
  });
}

int scvs_modes_to_keep(const double *incr2, int64_t n, double eps, int32_t patience, int64_t *n_keep) {
  if (!incr2 || !n_keep || n < 1 || patience < 1 || !(eps > 0)) return SCVS_ERR_ARG;
  *n_keep = n;
  for (int64_t N = 1; N + patience <= n; ++N) {
    bool small = true;
    for (int32_t q = 0; q < patience && small; ++q) small = std::sqrt(std::max(incr2[N + q], 0.0)) < eps;
    if (small) { *n_keep = N; break; }
  }
  return SCVS_OK;
}

int scvs_mesh_hash(int32_t dim, int64_t N, int64_t P, const double *xyz, int64_t E, const int32_t *conn,
                   const uint8_t *tag, uint64_t *hash) {
  if ((dim != 2 && dim != 3) || N <= 0 || P <= 0 || E <= 0 || !xyz || !conn || !tag || !hash) return SCVS_ERR_ARG;
  const int64_t sizes[4] = {dim, N, P, E};
  uint64_t h = fnv1a(FNV_OFFSET, sizes, sizeof(sizes));
  h = fnv1a(h, xyz, (size_t)N * dim * sizeof(double));
  h = fnv1a(h, conn, (size_t)E * (dim == 2 ? 6 : 10) * sizeof(int32_t));
  h = fnv1a(h, tag, (size_t)N);
  *hash = h;
  return SCVS_OK;
}

static int64_t ckpt_payload(const scvs_ckpt_header &h) {
  const int64_t m = h.n_modes;
  return m * (8 + 8 + 4 + 8) + m * h.n_nodes * h.dim * 16 + m * h.n_vertices * 16;
}

int scvs_data_hash(const scvs_c64 *g, int64_t n_g, const scvs_c64 *h, int64_t n_h, uint64_t *hash) {
  if (!hash || n_g < 0 || n_h < 0 || (n_g > 0 && !g) || (h && n_h < 0)) return SCVS_ERR_ARG;
  const int64_t sizes[2] = {n_g, h ? n_h : -1};
  uint64_t v = fnv1a(FNV_OFFSET, sizes, sizeof(sizes));
  if (n_g > 0) v = fnv1a(v, g, (size_t)n_g * sizeof(scvs_c64));
  if (h && n_h > 0) v = fnv1a(v, h, (size_t)n_h * sizeof(scvs_c64));
  *hash = v;
  return SCVS_OK;
}

static bool ckpt_header_ok(const scvs_ckpt_header &h) {
  return (h.dim == 2 || h.dim == 3) && h.n_modes >= 1 && h.n_modes <= 128 && h.n_nodes > 0 && h.n_vertices > 0 &&
         h.n_vertices <= h.n_nodes && h.n_nodes < INT32_MAX;
}

int scvs_checkpoint_write(const char *path, const scvs_ckpt_header *hd, const double *omega, const uint64_t *data_hash,
                          const int32_t *status, const double *rel_res, const scvs_c64 *u, const scvs_c64 *p) {
  if (!path || !hd || !omega || !data_hash || !status || !rel_res || !u || !p || !ckpt_header_ok(*hd))
    return SCVS_ERR_ARG;
  const scvs_ckpt_header &h = *hd;
  const int64_t m = h.n_modes, nu = (int64_t)h.n_nodes * h.dim;
  FILE *f = std::fopen(path, "wb");
  if (!f) return SCVS_ERR_ARG;
  uint64_t sum = FNV_OFFSET;
  bool ok = true;
  auto put = [&](const void *d, size_t n) {
    if (!ok) return;
    ok = std::fwrite(d, 1, n, f) == n;
    sum = fnv1a(sum, d, n);
  };
  put(CKPT_MAGIC, sizeof(CKPT_MAGIC));
  put(&h, sizeof(h));
  put(omega, m * sizeof(double));
  put(data_hash, m * sizeof(uint64_t));
  put(status, m * sizeof(int32_t));
  put(rel_res, m * sizeof(double));
  put(u, (size_t)m * nu * sizeof(scvs_c64));
  put(p, (size_t)m * h.n_vertices * sizeof(scvs_c64));
  if (ok) ok = std::fwrite(&sum, 1, sizeof(sum), f) == sizeof(sum);
  ok = (std::fclose(f) == 0) && ok;
  return ok ? SCVS_OK : SCVS_ERR_ARG;
}

int scvs_checkpoint_read(const char *path, scvs_ckpt_header *hd, double *omega, uint64_t *data_hash, int32_t *status,
                         double *rel_res, scvs_c64 *u, scvs_c64 *p) {
  if (!path || !hd) return SCVS_ERR_ARG;
  const bool fill = omega || data_hash || status || rel_res || u || p;
  const scvs_ckpt_header expect = *hd;  // the arrays' sizes when filling
  FILE *f = std::fopen(path, "rb");
  if (!f) return SCVS_ERR_ARG;
  std::vector<char> buf;
  char chunk[1 << 16];
  size_t n;
  while ((n = std::fread(chunk, 1, sizeof(chunk), f)) > 0) buf.insert(buf.end(), chunk, chunk + n);
  std::fclose(f);
  scvs_ckpt_header h{};
  const size_t head = sizeof(CKPT_MAGIC) + sizeof(h);
  if (buf.size() < head + sizeof(uint64_t) || std::memcmp(buf.data(), CKPT_MAGIC, sizeof(CKPT_MAGIC)) != 0)
    return SCVS_ERR_ARG;
  std::memcpy(&h, buf.data() + sizeof(CKPT_MAGIC), sizeof(h));
  if (!ckpt_header_ok(h) || (int64_t)buf.size() != (int64_t)head + ckpt_payload(h) + (int64_t)sizeof(uint64_t))
    return SCVS_ERR_ARG;
  uint64_t stored = 0;
  std::memcpy(&stored, buf.data() + buf.size() - sizeof(stored), sizeof(stored));
  if (fnv1a(FNV_OFFSET, buf.data(), buf.size() - sizeof(stored)) != stored) return SCVS_ERR_ARG;
  if (fill && (h.dim != expect.dim || h.n_modes != expect.n_modes || h.n_nodes != expect.n_nodes ||
               h.n_vertices != expect.n_vertices))
    return SCVS_ERR_ARG;  // the file no longer matches the header the caller sized its arrays for
  *hd = h;
  const int64_t m = h.n_modes, nu = (int64_t)h.n_nodes * h.dim;
  const char *q = buf.data() + head;
  auto take = [&](void *dst, size_t bytes) {
    if (dst) std::memcpy(dst, q, bytes);
    q += bytes;
  };
  take(omega, m * sizeof(double));
  take(data_hash, m * sizeof(uint64_t));
  take(status, m * sizeof(int32_t));
  take(rel_res, m * sizeof(double));
  take(u, (size_t)m * nu * sizeof(scvs_c64));
  take(p, (size_t)m * h.n_vertices * sizeof(scvs_c64));
  return SCVS_OK;
}

int scvs_graph_aggregates(int64_t n_vert, const int64_t *row_ptr, const int32_t *col, int32_t target,
                          int32_t *agg, int32_t *n_agg, int32_t *n_blk) {
  if (n_vert < 0 || n_vert > INT32_MAX || !row_ptr || !agg || target < 1 || target > 512) return SCVS_ERR_ARG;
  if (row_ptr[0] != 0) return SCVS_ERR_ARG;
  for (int64_t v = 0; v < n_vert; ++v)
    if (row_ptr[v + 1] < row_ptr[v]) return SCVS_ERR_ARG;
  if (row_ptr[n_vert] > 0 && !col) return SCVS_ERR_ARG;
  for (int64_t e = 0; e < row_ptr[n_vert]; ++e)
    if (col[e] < 0 || col[e] >= n_vert) return SCVS_ERR_ARG;
  try {
    const AggResult r = graph_aggregates(n_vert, row_ptr, col, target);
    std::copy(r.agg.begin(), r.agg.end(), agg);
    if (n_agg) *n_agg = (int32_t)r.blk.size();
    if (n_blk) *n_blk = r.n_blk;
  } catch (...) {
    return SCVS_ERR_OOM;
  }
  return SCVS_OK;
}

int scvs_schur_coarse_info(scvs_ctx *c, int32_t mesh_id, int32_t *info) {
  return guarded(c, [&]() {
    Mesh *m = get_mesh(c, mesh_id);
    if (!m || !info) return fail(c, SCVS_ERR_ARG, "bad mesh id or null info");
    const PcTables &t = m->pc;
    const bool built = t.cs_bytes != 0;
    info[0] = built ? t.n_agg : 0;
    info[1] = built ? t.n_blk : 0;
    info[2] = built ? t.na_max : 0;
    info[3] = built ? t.cs_singular : 0;
    return SCVS_OK;
  });
}

int scvs_lap_info(scvs_ctx *c, int32_t mesh_id, int32_t *info, int32_t *agg) {
  return guarded(c, [&]() {
    Mesh *m = get_mesh(c, mesh_id);
    if (!m || !info) return fail(c, SCVS_ERR_ARG, "bad mesh id or null info");
    const LapCoarse &L = m->lap;
    info[0] = L.on ? 1 : 0;
    info[1] = L.target ? L.n_agg : 0;
    info[2] = L.target ? L.n_blk : 0;
    info[3] = L.target ? L.na_max : 0;
    info[4] = L.target ? L.singular : 0;
    info[5] = L.target ? L.unanchored : 0;
    if (agg) {
      if (L.on) {
        SCVS_CUDA(cudaMemcpyAsync(agg, L.agg, m->P * sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
        SCVS_CUDA(cudaStreamSynchronize(c->stream));
      } else {
        std::fill(agg, agg + m->P, -1);
      }
    }
    return SCVS_OK;
  });
}

int scvs_pc_bounds(scvs_ctx *c, int32_t mesh_id, int32_t n_modes, double *out) {
  return guarded(c, [&]() {
    Mesh *m = get_mesh(c, mesh_id);
    if (!m || !out) return fail(c, SCVS_ERR_ARG, "bad mesh id or null out");
    if (m->m < 1 || (int)m->lam_u.size() < m->m) return fail(c, SCVS_ERR_STATE, "no modes set");
    if (n_modes != m->m) return fail(c, SCVS_ERR_ARG, "n_modes differs from the mesh's");
    out[0] = m->lam_m;
    out[1] = m->lam_l;
    for (int k = 0; k < n_modes; ++k) {
      out[2 + k] = m->lam_u[k];
      out[2 + n_modes + k] = m->lam_c[k];
    }
    return SCVS_OK;
  });
}

int scvs_kernel_timers(scvs_ctx *c, int32_t enable) {
  return guarded(c, [&]() {
    c->timers.reset();
    c->timers.on = enable != 0;
    return SCVS_OK;
  });
}

int scvs_kernel_times(scvs_ctx *c, int32_t n_classes, double *ms, double *bytes, int64_t *launches) {
  return guarded(c, [&]() {
    c->timers.resolve();
    for (int i = 0; i < n_classes && i < KC_COUNT; ++i) {
      if (ms) ms[i] = c->timers.ms[i];
      if (bytes) bytes[i] = c->timers.bytes[i];
      if (launches) launches[i] = c->timers.n[i];
    }
    return KC_COUNT;
  });
}

}  // extern "C"
