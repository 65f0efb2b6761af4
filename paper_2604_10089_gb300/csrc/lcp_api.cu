// C ABI of the collision-resolution library: context set-up (Sec. 3 of the
// paper: contacts, D, U_nc, b), mobility applications (Sec. 2) and the LCP
// solves (Algorithms 1 and 4).  All arithmetic runs in the kernels of the
// other translation units; this file validates arguments, owns memory and
// sequences the launches.
#include <cmath>
#include <cstring>
#include <new>

#include "common.cuh"

int stokes_configure(lcp_ctx* ctx);
int stokes_max_splits(const lcp_ctx* ctx);
int stokes_velocity(lcp_ctx* ctx, const double* phi, double* UO);
int pqn_configure(lcp_ctx* ctx, int rmax);

static thread_local std::string g_setup_error;

// b = gap / dt + D^T U_nc (Eq. defAandb)
__global__ void k_build_b(int n, double inv_dt, const double* gap, const double* dtu, double* b) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l < n) b[l] = gap[l] * inv_dt + dtu[l];
}

extern "C" void lcp_default_config(lcp_config* c) {
  if (!c) return;
  std::memset(c, 0, sizeof(*c));
  c->n_theta = 9;
  c->n_phi = 18;
  c->radius = 1.0;
  c->contact_radius = 1.25;
  c->viscosity = 1.0;
  c->dt = 0.01;
  c->delta = 0.05;
  c->precision = LCP_FP64;
  c->gmres_tol = 1e-12;
  c->gmres_restart = 60;
  c->gmres_maxit = 600;
  c->inner_tol = 1e-5;
  c->ir_maxit = 8;
  c->kmax = 100;
  c->kmax_inner = 100;
  c->memory = 32;
  c->ssn_maxit = 50;
  c->forcing = 1e-3;
  c->cuda_stream = nullptr;
}

static int validate(const lcp_config* c, int M, const double* centers, std::string* err) {
  if (!c) { *err = "config is NULL"; return LCP_ERR_INVALID_ARG; }
  if (M < 1 || !centers) { *err = "need at least one body and its centre"; return LCP_ERR_INVALID_ARG; }
  if (c->n_theta < 2 || c->n_phi < 4 || (c->n_phi & 1)) { *err = "grid needs n_theta >= 2 and an even n_phi >= 4"; return LCP_ERR_INVALID_ARG; }
  if (c->n_theta * c->n_phi > 512) { *err = "at most 512 nodes per sphere"; return LCP_ERR_INVALID_ARG; }
  if (!(c->radius > 0) || !(c->viscosity > 0) || !(c->dt > 0) || !(c->contact_radius >= c->radius)) {
    *err = "radius, viscosity, dt must be positive and contact_radius >= radius";
    return LCP_ERR_INVALID_ARG;
  }
  if (c->precision != LCP_FP64 && c->precision != LCP_MIXED) { *err = "precision must be LCP_FP64 or LCP_MIXED"; return LCP_ERR_INVALID_ARG; }
  if (c->gmres_restart < 1 || c->gmres_restart > 200 || c->gmres_maxit < 1) { *err = "gmres_restart in [1, 200], gmres_maxit >= 1"; return LCP_ERR_INVALID_ARG; }
  if (c->memory < 1 || c->memory > 60) { *err = "memory in [1, 60]"; return LCP_ERR_INVALID_ARG; }
  if (c->kmax < 1 || c->kmax > 120 || c->kmax_inner < 1) { *err = "kmax in [1, 120], kmax_inner >= 1"; return LCP_ERR_INVALID_ARG; }
  if (!(c->gmres_tol > 0) || !(c->inner_tol > 0) || c->ir_maxit < 1 || c->ssn_maxit < 1) { *err = "tolerances and iteration limits must be positive"; return LCP_ERR_INVALID_ARG; }
  for (int i = 0; i < 3 * M; i++)
    if (!std::isfinite(centers[i])) { *err = "non-finite centre coordinate"; return LCP_ERR_INVALID_ARG; }
  return LCP_OK;
}

static int setup_impl(lcp_ctx* ctx, const double* centers, const double* axes, int n_contacts,
                      const lcp_contact* contacts) {
  const int M = ctx->M;
  ctx->centers = (double*)ctx_alloc(ctx, sizeof(double) * 3 * M);
  if (!ctx->centers) return LCP_ERR_OOM;
  LCP_CUDA(cudaMemcpyAsync(ctx->centers, centers, sizeof(double) * 3 * M, cudaMemcpyHostToDevice, ctx->stream));
  if (axes) {
    ctx->axes = (double*)ctx_alloc(ctx, sizeof(double) * 3 * M);
    if (!ctx->axes) return LCP_ERR_OOM;
    LCP_CUDA(cudaMemcpyAsync(ctx->axes, axes, sizeof(double) * 3 * M, cudaMemcpyHostToDevice, ctx->stream));
  }
  LCP_TRY(geometry_build(ctx));
  if (contacts) {
    LCP_TRY(contacts_upload(ctx, n_contacts, contacts));
    ctx->n = n_contacts;
  } else {
    LCP_TRY(contacts_detect(ctx, &ctx->n));
  }
  LCP_TRY(contacts_csr(ctx));
  const int N = ctx->N, n = ctx->n, L = 3 * N;
  ctx->m = ctx->cfg.gmres_restart;
  ctx->splits = stokes_max_splits(ctx);
  ctx->dot_blocks = 2 * 152;
  ctx->V = (double*)ctx_alloc(ctx, sizeof(double) * (size_t)L * (ctx->m + 1));
  ctx->H = (double*)ctx_alloc(ctx, sizeof(double) * ((size_t)(ctx->m + 1) * ctx->m + 6 * (size_t)ctx->m + 16));
  ctx->phi = (double*)ctx_alloc(ctx, sizeof(double) * L);
  ctx->rhs = (double*)ctx_alloc(ctx, sizeof(double) * L);
  ctx->res = (double*)ctx_alloc(ctx, sizeof(double) * L);
  ctx->wv = (double*)ctx_alloc(ctx, sizeof(double) * L);
  ctx->dphi = (double*)ctx_alloc(ctx, sizeof(double) * L);
  ctx->phi32 = (float*)ctx_alloc(ctx, sizeof(float) * L);
  ctx->partial = (double*)ctx_alloc(ctx, sizeof(double) * (size_t)L * ctx->splits);
  ctx->coef = (double*)ctx_alloc(ctx, sizeof(double) * 6 * M);
  ctx->dotp = (double*)ctx_alloc(ctx, sizeof(double) * (size_t)(ctx->m + 2) * ctx->dot_blocks);
  ctx->FT = (double*)ctx_alloc(ctx, sizeof(double) * 6 * M);
  ctx->UO = (double*)ctx_alloc(ctx, sizeof(double) * 6 * M);
  ctx->U_nc = (double*)ctx_alloc(ctx, sizeof(double) * 6 * M);
  ctx->dscal = (double*)ctx_alloc(ctx, sizeof(double) * 64);
  ctx->b = (double*)ctx_alloc(ctx, sizeof(double) * (n > 0 ? n : 1));
  ctx->tmp_n = (double*)ctx_alloc(ctx, sizeof(double) * (n > 0 ? n : 1));
  ctx->tmp_n2 = (double*)ctx_alloc(ctx, sizeof(double) * (n > 0 ? n : 1));
  ctx->tmp_n3 = (double*)ctx_alloc(ctx, sizeof(double) * (n > 0 ? n : 1));
  ctx->Uh = (double*)ctx_alloc(ctx, sizeof(double) * (size_t)(n > 0 ? n : 1) * ctx->cfg.kmax);
  ctx->Vh = (double*)ctx_alloc(ctx, sizeof(double) * (size_t)(n > 0 ? n : 1) * ctx->cfg.kmax);
  if (!ctx->V || !ctx->H || !ctx->phi || !ctx->rhs || !ctx->res || !ctx->wv || !ctx->dphi || !ctx->phi32 ||
      !ctx->partial || !ctx->coef || !ctx->dotp || !ctx->FT || !ctx->UO || !ctx->U_nc || !ctx->dscal || !ctx->b ||
      !ctx->tmp_n || !ctx->tmp_n2 || !ctx->tmp_n3 || !ctx->Uh || !ctx->Vh) {
    ctx->err = "device allocation failed";
    return LCP_ERR_OOM;
  }
  LCP_CUDA(cudaMallocHost((void**)&ctx->hscal, sizeof(double) * 64));
  LCP_CUDA(cudaMemsetAsync(ctx->dscal, 0, sizeof(double) * 64, ctx->stream));
  LCP_TRY(pqn_alloc(ctx, &ctx->pq_outer, n, ctx->cfg.memory));
  LCP_TRY(pqn_alloc(ctx, &ctx->pq_inner, n, ctx->cfg.memory));
  LCP_TRY(stokes_configure(ctx));
  LCP_TRY(pqn_configure(ctx, ctx->cfg.memory));
  // U_nc: slip-driven velocities with F = T = 0
  LCP_CUDA(cudaMemsetAsync(ctx->FT, 0, sizeof(double) * 6 * M, ctx->stream));
  if (ctx->axes) {
    LCP_TRY(mobility_solve(ctx, ctx->FT, 1, ctx->U_nc));
  } else {
    LCP_CUDA(cudaMemsetAsync(ctx->U_nc, 0, sizeof(double) * 6 * M, ctx->stream));
  }
  if (n > 0) {
    LCP_TRY(gather_Dt(ctx, ctx->U_nc, ctx->tmp_n, nullptr));
    k_build_b<<<(n + 127) / 128, 128, 0, ctx->stream>>>(n, 1.0 / ctx->cfg.dt, ctx->gap, ctx->tmp_n, ctx->b);
    LCP_CUDA(cudaGetLastError());
  }
  LCP_CUDA(cudaStreamSynchronize(ctx->stream));
  return LCP_OK;
}

extern "C" int lcp_setup(const lcp_config* cfg, int n_bodies, const double* centers, const double* axes,
                         int n_contacts, const lcp_contact* contacts, lcp_ctx** out) {
  if (!out) { g_setup_error = "out is NULL"; return LCP_ERR_INVALID_ARG; }
  *out = nullptr;
  std::string err;
  int st = validate(cfg, n_bodies, centers, &err);
  if (st == LCP_OK && contacts && n_contacts < 0) { err = "negative contact count"; st = LCP_ERR_INVALID_ARG; }
  if (st != LCP_OK) { g_setup_error = err; return st; }
  lcp_ctx* ctx = new (std::nothrow) lcp_ctx();
  if (!ctx) { g_setup_error = "host allocation failed"; return LCP_ERR_OOM; }
  ctx->cfg = *cfg;
  ctx->stream = (cudaStream_t)cfg->cuda_stream;
  ctx->M = n_bodies;
  ctx->ns = cfg->n_theta * cfg->n_phi;
  ctx->N = ctx->M * ctx->ns;
  st = setup_impl(ctx, centers, axes, n_contacts, contacts);
  if (st != LCP_OK) {
    g_setup_error = ctx->err.empty() ? std::string("setup failed") : ctx->err;
    lcp_destroy(ctx);
    return st;
  }
  *out = ctx;
  return LCP_OK;
}

extern "C" void lcp_destroy(lcp_ctx* ctx) {
  if (!ctx) return;
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  else cudaDeviceSynchronize();
  for (void* p : ctx->allocs) cudaFree(p);
  if (ctx->hscal) cudaFreeHost(ctx->hscal);
  delete ctx;
}

extern "C" const char* lcp_last_error(const lcp_ctx* ctx) {
  return ctx ? ctx->err.c_str() : g_setup_error.c_str();
}

extern "C" int lcp_sizes(const lcp_ctx* ctx, int* n_bodies, int* n_nodes, int* n_contacts) {
  if (!ctx) return LCP_ERR_INVALID_ARG;
  if (n_bodies) *n_bodies = ctx->M;
  if (n_nodes) *n_nodes = ctx->N;
  if (n_contacts) *n_contacts = ctx->n;
  return LCP_OK;
}

extern "C" int lcp_get_contacts(lcp_ctx* ctx, lcp_contact* out) {
  if (!ctx || (!out && ctx->n)) return LCP_ERR_INVALID_ARG;
  const int n = ctx->n;
  if (n == 0) return LCP_OK;
  std::vector<int> hi(n), hj(n);
  std::vector<double> hn(3 * (size_t)n), hg(n);
  LCP_CUDA(cudaMemcpyAsync(hi.data(), ctx->ci, sizeof(int) * n, cudaMemcpyDeviceToHost, ctx->stream));
  LCP_CUDA(cudaMemcpyAsync(hj.data(), ctx->cj, sizeof(int) * n, cudaMemcpyDeviceToHost, ctx->stream));
  LCP_CUDA(cudaMemcpyAsync(hn.data(), ctx->cnrm, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, ctx->stream));
  LCP_CUDA(cudaMemcpyAsync(hg.data(), ctx->gap, sizeof(double) * n, cudaMemcpyDeviceToHost, ctx->stream));
  LCP_CUDA(cudaStreamSynchronize(ctx->stream));
  for (int l = 0; l < n; l++) {
    out[l].i = hi[l];
    out[l].j = hj[l];
    for (int d = 0; d < 3; d++) out[l].normal[d] = hn[3 * l + d];
    out[l].gap = hg[l];
  }
  return LCP_OK;
}

static int copy_out(lcp_ctx* ctx, double* host, const double* dev, size_t count) {
  if (count == 0) return LCP_OK;
  if (!host) { ctx->err = "output pointer is NULL"; return LCP_ERR_INVALID_ARG; }
  LCP_CUDA(cudaMemcpyAsync(host, dev, sizeof(double) * count, cudaMemcpyDeviceToHost, ctx->stream));
  LCP_CUDA(cudaStreamSynchronize(ctx->stream));
  return LCP_OK;
}

extern "C" int lcp_get_b(lcp_ctx* ctx, double* b) {
  if (!ctx) return LCP_ERR_INVALID_ARG;
  return copy_out(ctx, b, ctx->b, ctx->n);
}

extern "C" int lcp_get_unc(lcp_ctx* ctx, double* u) {
  if (!ctx) return LCP_ERR_INVALID_ARG;
  return copy_out(ctx, u, ctx->U_nc, 6 * (size_t)ctx->M);
}

static int mobility_impl(lcp_ctx* ctx, const double* FT, double* UO, int include_slip, int fidelity) {
  if (include_slip && !ctx->axes) { ctx->err = "no Janus axes were given at set-up"; return LCP_ERR_INVALID_ARG; }
  if (fidelity == LCP_HIGH) {
    return mobility_solve(ctx, FT, include_slip, UO);
  } else if (fidelity == LCP_LOW_RPY) {
    if (include_slip) { ctx->err = "the RPY operator has no slip term"; return LCP_ERR_INVALID_ARG; }
    return rpy_apply(ctx, FT, UO);
  }
  ctx->err = "unknown fidelity";
  return LCP_ERR_INVALID_ARG;
}

extern "C" int mobility_apply_dev(lcp_ctx* ctx, const double* FT, double* UO, int include_slip, int fidelity) {
  if (!ctx || !FT || !UO) return LCP_ERR_INVALID_ARG;
  LCP_TRY(mobility_impl(ctx, FT, UO, include_slip, fidelity));
  LCP_CUDA(cudaStreamSynchronize(ctx->stream));
  return LCP_OK;
}

extern "C" int mobility_apply(lcp_ctx* ctx, const double* FT, double* UO, int include_slip, int fidelity) {
  if (!ctx || !FT || !UO) return LCP_ERR_INVALID_ARG;
  const int M = ctx->M;
  double* fdev = ctx->FT;
  LCP_CUDA(cudaMemcpyAsync(fdev, FT, sizeof(double) * 6 * M, cudaMemcpyHostToDevice, ctx->stream));
  LCP_TRY(mobility_impl(ctx, fdev, ctx->UO, include_slip, fidelity));
  return copy_out(ctx, UO, ctx->UO, 6 * (size_t)M);
}

extern "C" int lcp_apply_A(lcp_ctx* ctx, const double* x, double* Ax, int fidelity) {
  if (!ctx || (ctx->n && (!x || !Ax))) return LCP_ERR_INVALID_ARG;
  if (ctx->n == 0) return LCP_OK;
  LCP_CUDA(cudaMemcpyAsync(ctx->tmp_n2, x, sizeof(double) * ctx->n, cudaMemcpyHostToDevice, ctx->stream));
  if (fidelity == LCP_HIGH) {
    LCP_TRY(mvp_high(ctx, ctx->tmp_n2, ctx->tmp_n3));
  } else if (fidelity == LCP_LOW_RPY) {
    LCP_TRY(mvp_low(ctx, ctx->tmp_n2, ctx->tmp_n3));
  } else {
    ctx->err = "unknown fidelity";
    return LCP_ERR_INVALID_ARG;
  }
  return copy_out(ctx, Ax, ctx->tmp_n3, ctx->n);
}

extern "C" int lcp_solve_dev(lcp_ctx* ctx, int method, double tol, const double* x0, double* x, lcp_stats* st) {
  if (!ctx || (ctx->n && !x) || !(tol >= 0.0)) return LCP_ERR_INVALID_ARG;
  if (method != LCP_MONO_PQN && method != LCP_BI_PQN) { ctx->err = "unknown method"; return LCP_ERR_INVALID_ARG; }
  return lcp_solve_device(ctx, method, tol, x0, x, st);
}

extern "C" int lcp_solve(lcp_ctx* ctx, int method, double tol, const double* x0, double* x, lcp_stats* st) {
  if (!ctx || (ctx->n && !x) || !(tol >= 0.0)) return LCP_ERR_INVALID_ARG;
  if (method != LCP_MONO_PQN && method != LCP_BI_PQN) { ctx->err = "unknown method"; return LCP_ERR_INVALID_ARG; }
  const int n = ctx->n;
  const double* x0d = nullptr;
  if (x0 && n) {
    LCP_CUDA(cudaMemcpyAsync(ctx->tmp_n2, x0, sizeof(double) * n, cudaMemcpyHostToDevice, ctx->stream));
    x0d = ctx->tmp_n2;
  }
  const int status = lcp_solve_device(ctx, method, tol, x0d, ctx->tmp_n3, st);
  if (status != LCP_OK && status != LCP_ERR_NOT_CONVERGED) return status;
  LCP_TRY(copy_out(ctx, x, ctx->tmp_n3, n));
  return status;
}

extern "C" int lcp_stokes_apply_dev(lcp_ctx* ctx, const double* phi, double* out, int precision) {
  if (!ctx || !phi || !out) return LCP_ERR_INVALID_ARG;
  if (precision != LCP_FP64 && precision != LCP_MIXED) return LCP_ERR_INVALID_ARG;
  LCP_TRY(stokes_apply(ctx, phi, out, precision));
  LCP_CUDA(cudaStreamSynchronize(ctx->stream));
  return LCP_OK;
}

extern "C" int lcp_stokes_rhs_dev(lcp_ctx* ctx, const double* FT, int include_slip, double* rhs) {
  if (!ctx || !FT || !rhs) return LCP_ERR_INVALID_ARG;
  if (include_slip && !ctx->axes) { ctx->err = "no Janus axes were given at set-up"; return LCP_ERR_INVALID_ARG; }
  LCP_TRY(stokes_rhs(ctx, FT, include_slip, rhs));
  LCP_CUDA(cudaStreamSynchronize(ctx->stream));
  return LCP_OK;
}

extern "C" int lcp_rigid_velocity_dev(lcp_ctx* ctx, const double* phi, double* UO) {
  if (!ctx || !phi || !UO) return LCP_ERR_INVALID_ARG;
  LCP_TRY(stokes_velocity(ctx, phi, UO));
  LCP_CUDA(cudaStreamSynchronize(ctx->stream));
  return LCP_OK;
}
