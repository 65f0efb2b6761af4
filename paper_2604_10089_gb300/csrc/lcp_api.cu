// C ABI of the collision-resolution library: context set-up (Sec. 3 of the
// paper: contacts, D, U_nc, b), mobility applications (Sec. 2) and the LCP
// solves (Algorithms 1 and 4).  All arithmetic runs in the kernels of the
// other translation units; this file validates arguments, owns memory and
// sequences the launches.
#include <cmath>
#include <cstring>
#include <algorithm>
#include <new>

#include "common.cuh"

int stokes_configure(lcp_ctx* ctx);
int stokes_max_splits(const lcp_ctx* ctx);
int stokes_sym_configure(lcp_ctx* ctx);
size_t stokes_sym_bytes(int M, int ns);
int stokes_select_variant(lcp_ctx* ctx, const char* name);
int stokes_velocity(lcp_ctx* ctx, const double* phi, double* UO);
int pqn_configure(lcp_ctx* ctx, int rmax);
int stokes_autotune(lcp_ctx* ctx);
const char* stokes_variant_name(const lcp_ctx* ctx);

static thread_local std::string g_setup_error;
static int copy_out(lcp_ctx* ctx, double* host, const double* dev, size_t count);

void lcp_set_thread_error(const std::string& msg) { g_setup_error = msg; }

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
  c->inner_tol = 1e-6;
  c->ir_maxit = 8;
  c->kmax = 100;
  c->kmax_inner = 100;
  c->memory = 32;
  c->lowfi_n_theta = 0;
  c->lowfi_n_phi = 0;
  c->lowfi_tol = 1e-6;
  c->init_forcing = 0.0;
  c->ssn_maxit = 50;
  c->forcing = 1e-3;
  c->precondition = 1;
  c->residual_precision = LCP_DF64;
  c->autotune = 0;
  c->own_stream = 0;
  c->h0_scaling = 1;
  c->warm_start = LCP_WARM_FORCES;
  c->recycle = 0;
  c->self_quadrature = 1;
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
  if (c->residual_precision != LCP_FP64 && c->residual_precision != LCP_DF64) { *err = "residual_precision must be LCP_FP64 or LCP_DF64"; return LCP_ERR_INVALID_ARG; }
  if (c->gmres_restart < 1 || c->gmres_restart > 200 || c->gmres_maxit < 1) { *err = "gmres_restart in [1, 200], gmres_maxit >= 1"; return LCP_ERR_INVALID_ARG; }
  if (c->lowfi_n_theta != 0 && (c->lowfi_n_theta < 2 || c->lowfi_n_phi < 4 || (c->lowfi_n_phi & 1) ||
                                 (size_t)c->lowfi_n_theta * c->lowfi_n_phi > 512 || !(c->lowfi_tol > 0.0) ||
                                 c->lowfi_tol > 0.1)) {
    *err = "low-fidelity grid: lowfi_n_theta >= 2, even lowfi_n_phi >= 4, at most 512 nodes, lowfi_tol in (0, 0.1]";
    return LCP_ERR_INVALID_ARG;
  }
  if (c->warm_start < 0 || c->warm_start > (LCP_WARM_SLIP | LCP_WARM_FORCES | LCP_WARM_NO_INIT)) { *err = "warm_start: a combination of the LCP_WARM_* flags"; return LCP_ERR_INVALID_ARG; }
  if (c->self_quadrature != 0 && c->self_quadrature != 1) { *err = "self_quadrature must be 0 or 1"; return LCP_ERR_INVALID_ARG; }
  if (c->recycle < 0 || c->recycle > c->gmres_restart) { *err = "recycle in [0, gmres_restart]"; return LCP_ERR_INVALID_ARG; }
  if (!(c->init_forcing >= 0.0) || c->init_forcing >= 1.0) { *err = "init_forcing in [0, 1)"; return LCP_ERR_INVALID_ARG; }
  // the direction kernel keeps its r x r systems in shared memory (<= 227 KB: r <= 48)
  if (c->memory < 1 || c->memory > 48) { *err = "memory in [1, 48]"; return LCP_ERR_INVALID_ARG; }
  if (c->kmax < 1 || c->kmax > 120 || c->kmax_inner < 1) { *err = "kmax in [1, 120], kmax_inner >= 1"; return LCP_ERR_INVALID_ARG; }
  if (!(c->gmres_tol > 0) || !(c->inner_tol > 0) || c->ir_maxit < 1 || c->ssn_maxit < 1) { *err = "tolerances and iteration limits must be positive"; return LCP_ERR_INVALID_ARG; }
  for (int i = 0; i < 3 * M; i++)
    if (!std::isfinite(centers[i])) { *err = "non-finite centre coordinate"; return LCP_ERR_INVALID_ARG; }
  return LCP_OK;
}

static int alloc_static(lcp_ctx* ctx);

// The coarse-grid context of the low-fidelity operator: same bodies and
// stream, grid lowfi_n_theta x lowfi_n_phi, FP32-operator GMRES to lowfi_tol,
// no contacts or quasi-Newton state of its own.  Owned by ctx.
static int lowfi_create(lcp_ctx* ctx) {
  lcp_ctx* lo = new (std::nothrow) lcp_ctx();
  if (!lo) { ctx->err = "host allocation failed"; return LCP_ERR_OOM; }
  lo->cfg = ctx->cfg;
  lo->cfg.n_theta = ctx->cfg.lowfi_n_theta;
  lo->cfg.n_phi = ctx->cfg.lowfi_n_phi;
  lo->cfg.precision = LCP_MIXED;
  lo->cfg.gmres_tol = ctx->cfg.lowfi_tol;
  lo->cfg.memory = 1;
  lo->cfg.own_stream = 0;
  lo->cfg.lowfi_n_theta = 0;
  lo->cfg.lowfi_n_phi = 0;
  // the kernel choice follows the parent's autotune setting; by default the
  // size rule picks it, which keeps the choice independent of timing noise
  // (and of a profiler's launch overhead)
  lo->stream = ctx->stream;
  lo->device = ctx->device;
  lo->M = ctx->M;
  lo->ns = lo->cfg.n_theta * lo->cfg.n_phi;
  lo->N = lo->M * lo->ns;
  lo->fp32_only = true;
  ctx->lo = lo;
  const int st = alloc_static(lo);
  if (st != LCP_OK) ctx->err = "low-fidelity grid: " + lo->err;
  return st;
}

// Buffers whose size depends only on M and the grid (once per context).
static int alloc_static(lcp_ctx* ctx) {
  const int M = ctx->M, N = ctx->N, L = 3 * N;
  ctx->centers = (double*)ctx_alloc(ctx, sizeof(double) * 3 * M);
  ctx->axes = (double*)ctx_alloc(ctx, sizeof(double) * 3 * M);
  ctx->dscal = (double*)ctx_alloc(ctx, sizeof(double) * 64);
  if (!ctx->centers || !ctx->axes || !ctx->dscal) return LCP_ERR_OOM;
  LCP_CUDA(cudaMallocHost((void**)&ctx->hscal, sizeof(double) * 64));
  LCP_CUDA(cudaMemsetAsync(ctx->dscal, 0, sizeof(double) * 64, ctx->stream));
  LCP_TRY(geometry_build(ctx));
  ctx->m = ctx->cfg.gmres_restart;
  LCP_TRY(stokes_configure(ctx));
  LCP_TRY(stokes_sym_configure(ctx));
  ctx->splits = std::max(stokes_max_splits(ctx), ctx->sym_slots);
  ctx->dot_blocks = 2 * 152;
  ctx->V = (double*)ctx_alloc(ctx, sizeof(double) * (size_t)L * (ctx->m + 1));
  if (ctx->cfg.precondition) {
    ctx->Z = (double*)ctx_alloc(ctx, sizeof(double) * (size_t)L * ctx->m);
    if (!ctx->Z) return LCP_ERR_OOM;
  }
  ctx->H = (double*)ctx_alloc(ctx, sizeof(double) * ((size_t)(ctx->m + 1) * ctx->m + 6 * (size_t)ctx->m + 16));
  ctx->phi = (double*)ctx_alloc(ctx, sizeof(double) * L);
  ctx->rhs = (double*)ctx_alloc(ctx, sizeof(double) * L);
  ctx->res = (double*)ctx_alloc(ctx, sizeof(double) * L);
  ctx->wv = (double*)ctx_alloc(ctx, sizeof(double) * L);
  ctx->dphi = (double*)ctx_alloc(ctx, sizeof(double) * L);
  ctx->phi32 = (float*)ctx_alloc(ctx, sizeof(float) * L);
  ctx->phidf = (float*)ctx_alloc(ctx, sizeof(float) * 2 * L);
  ctx->partial = (double*)ctx_alloc(ctx, sizeof(double) * (size_t)L * ctx->splits);
  ctx->coef = (double*)ctx_alloc(ctx, sizeof(double) * 6 * M);
  ctx->dotp = (double*)ctx_alloc(ctx, sizeof(double) * (size_t)(ctx->m + 2) * ctx->dot_blocks);
  ctx->FT = (double*)ctx_alloc(ctx, sizeof(double) * 6 * M);
  ctx->UO = (double*)ctx_alloc(ctx, sizeof(double) * 6 * M);
  ctx->U_nc = (double*)ctx_alloc(ctx, sizeof(double) * 6 * M);
  ctx->phi_unc = (double*)ctx_alloc(ctx, sizeof(double) * L);
  ctx->rc_max = ctx->cfg.recycle;
  if (ctx->rc_max > 0) {
    ctx->rc_psi = (double*)ctx_alloc(ctx, sizeof(double) * (size_t)L * ctx->rc_max);
    ctx->rc_w = (double*)ctx_alloc(ctx, sizeof(double) * (size_t)L * ctx->rc_max);
    ctx->rc_h = (double*)ctx_alloc(ctx, sizeof(double) * 3 * ctx->rc_max);
    ctx->rc_phi0 = (double*)ctx_alloc(ctx, sizeof(double) * L);
    ctx->rc_r0 = (double*)ctx_alloc(ctx, sizeof(double) * L);
    if (!ctx->rc_psi || !ctx->rc_w || !ctx->rc_h || !ctx->rc_phi0 || !ctx->rc_r0) return LCP_ERR_OOM;
  }
  ctx->MDx = (double*)ctx_alloc(ctx, sizeof(double) * 6 * M);
  ctx->cnext = (double*)ctx_alloc(ctx, sizeof(double) * 3 * M);
  ctx->anext = (double*)ctx_alloc(ctx, sizeof(double) * 3 * M);
  if (!ctx->MDx || !ctx->cnext || !ctx->anext) return LCP_ERR_OOM;
  if (!ctx->V || !ctx->H || !ctx->phi || !ctx->rhs || !ctx->res || !ctx->wv || !ctx->dphi || !ctx->phi32 ||
      !ctx->partial || !ctx->coef || !ctx->dotp || !ctx->FT || !ctx->UO || !ctx->U_nc || !ctx->phi_unc || !ctx->phidf) {
    ctx->err = "device allocation failed";
    return LCP_ERR_OOM;
  }
  if (ctx->cfg.self_quadrature) {   // before the preconditioner, which includes it
    LCP_TRY(self_correction_build(ctx));
    LCP_TRY(block_apply_reserve(ctx));
  }
  LCP_TRY(pqn_configure(ctx, ctx->cfg.memory));
  if (ctx->cfg.precondition) LCP_TRY(precond_build(ctx));
  if (ctx->cfg.autotune) LCP_TRY(stokes_autotune(ctx));
  if (ctx->cfg.lowfi_n_theta > 0) LCP_TRY(lowfi_create(ctx));
  return LCP_OK;
}

static size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }

// Contact-sized buffers (b, CSR entries, PQN states, high-fidelity corrections)
// in one arena, re-created only when n exceeds its capacity.
static int arena_ensure(lcp_ctx* ctx, int n) {
  if (ctx->arena && n <= ctx->ncap) return LCP_OK;
  int cap = ctx->ncap * 2;
  if (cap < n) cap = n;
  if (cap < 64) cap = 64;
  if (cap > ctx->pair_cap) cap = ctx->pair_cap > n ? ctx->pair_cap : n;
  const int R = ctx->cfg.memory, K = ctx->cfg.kmax;
  const size_t nn = cap;
  const size_t bytes = 4 * al256(sizeof(double) * nn) + al256(sizeof(int) * (2 * nn + 1)) +
                       2 * al256(sizeof(double) * nn * K) + 2 * pqn_bytes(cap, R);
  if (ctx->arena) {
    LCP_CUDA(cudaStreamSynchronize(ctx->stream));
    cudaFree(ctx->arena);
    ctx->arena = nullptr;
    ctx->ncap = 0;
    ctx->bytes -= ctx->arena_bytes;
    ctx->arena_bytes = 0;
  }
  if (cudaMalloc(&ctx->arena, bytes) != cudaSuccess) {
    cudaGetLastError();
    ctx->arena = nullptr;
    ctx->err = "device allocation of the contact buffers failed";
    return LCP_ERR_OOM;
  }
  ctx->arena_bytes = bytes;
  ctx->bytes += bytes;
  char* p = (char*)ctx->arena;
  ctx->b = (double*)p; p += al256(sizeof(double) * nn);
  ctx->tmp_n = (double*)p; p += al256(sizeof(double) * nn);
  ctx->tmp_n2 = (double*)p; p += al256(sizeof(double) * nn);
  ctx->tmp_n3 = (double*)p; p += al256(sizeof(double) * nn);
  ctx->bc_idx = (int*)p; p += al256(sizeof(int) * (2 * nn + 1));
  ctx->Uh = (double*)p; p += al256(sizeof(double) * nn * K);
  ctx->Vh = (double*)p; p += al256(sizeof(double) * nn * K);
  p = pqn_carve(&ctx->pq_outer, p, cap, R);
  p = pqn_carve(&ctx->pq_inner, p, cap, R);
  ctx->ncap = cap;
  return LCP_OK;
}

// Everything that depends on the configuration: centres (and axes), the
// collisional set and D, U_nc and b (Sec. 3, Eqs. collisional-set, defAandb).
// warm: start the slip solve from the previous slip density (time stepping).
static int configure(lcp_ctx* ctx, const double* centers, const double* axes, int n_contacts,
                     const lcp_contact* contacts, bool device_inputs, bool warm = false) {
  const int M = ctx->M;
  const cudaMemcpyKind kind = device_inputs ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  recycle_reset(ctx);   // K + P changes with the configuration
  ctx->x_warm_valid = false;
  LCP_CUDA(cudaMemcpyAsync(ctx->centers, centers, sizeof(double) * 3 * M, kind, ctx->stream));
  ctx->has_axes = axes != nullptr;
  if (axes) LCP_CUDA(cudaMemcpyAsync(ctx->axes, axes, sizeof(double) * 3 * M, kind, ctx->stream));
  LCP_TRY(geometry_update(ctx));
  if (ctx->lo) {
    LCP_CUDA(cudaMemcpyAsync(ctx->lo->centers, ctx->centers, sizeof(double) * 3 * M, cudaMemcpyDeviceToDevice,
                             ctx->stream));
    ctx->lo->has_axes = false;
    const int st = geometry_update(ctx->lo);
    if (st != LCP_OK) { ctx->err = "low-fidelity grid: " + ctx->lo->err; return st; }
  }
  if (contacts) {
    LCP_TRY(contacts_upload(ctx, n_contacts, contacts));
    ctx->n = n_contacts;
  } else {
    LCP_TRY(contacts_detect(ctx, &ctx->n));
  }
  const int n = ctx->n;
  LCP_TRY(arena_ensure(ctx, n));
  ctx->pq_outer.n = n;
  ctx->pq_inner.n = n;
  LCP_TRY(pqn_reset(ctx, &ctx->pq_outer));
  LCP_TRY(pqn_reset(ctx, &ctx->pq_inner));
  LCP_TRY(contacts_csr(ctx));
  // U_nc: slip-driven velocities with F = T = 0
  LCP_CUDA(cudaMemsetAsync(ctx->FT, 0, sizeof(double) * 6 * M, ctx->stream));
  ctx->unc_its = 0;
  ctx->unc_warm = 0;
  if (ctx->has_axes) {
    const bool use_warm = warm && (ctx->cfg.warm_start & LCP_WARM_SLIP) && ctx->phi_unc_valid;
    const int g0 = ctx->c_gmres;
    LCP_TRY(mobility_solve(ctx, ctx->FT, 1, ctx->U_nc, use_warm ? ctx->phi_unc : nullptr));
    ctx->unc_its = ctx->c_gmres - g0;
    ctx->unc_warm = use_warm ? 1 : 0;
    LCP_CUDA(cudaMemcpyAsync(ctx->phi_unc, ctx->phi, sizeof(double) * 3 * ctx->N, cudaMemcpyDeviceToDevice,
                             ctx->stream));
    ctx->phi_unc_valid = true;
  } else {
    LCP_CUDA(cudaMemsetAsync(ctx->U_nc, 0, sizeof(double) * 6 * M, ctx->stream));
    ctx->phi_unc_valid = false;
  }
  if (n > 0) {
    LCP_TRY(gather_Dt(ctx, ctx->U_nc, ctx->tmp_n, nullptr));
    ++ctx->nlaunch, k_build_b<<<(n + 127) / 128, 128, 0, ctx->stream>>>(n, 1.0 / ctx->cfg.dt, ctx->gap, ctx->tmp_n, ctx->b);
    LCP_CUDA(cudaGetLastError());
  }
  LCP_CUDA(cudaStreamSynchronize(ctx->stream));
  return LCP_OK;
}

static int setup_impl(lcp_ctx* ctx, const double* centers, const double* axes, int n_contacts,
                      const lcp_contact* contacts) {
  LCP_TRY(alloc_static(ctx));
  return configure(ctx, centers, axes, n_contacts, contacts, false);
}

static int check_finite(lcp_ctx* ctx, const double* c, int count) {
  for (int i = 0; i < count; i++)
    if (!std::isfinite(c[i])) { ctx->err = "non-finite input coordinate"; return LCP_ERR_INVALID_ARG; }
  return LCP_OK;
}

extern "C" int lcp_update(lcp_ctx* ctx, const double* centers, const double* axes, int n_contacts,
                          const lcp_contact* contacts) {
  if (!ctx || !centers) return LCP_ERR_INVALID_ARG;
  if (contacts && n_contacts < 0) { ctx->err = "negative contact count"; return LCP_ERR_INVALID_ARG; }
  LCP_TRY(check_finite(ctx, centers, 3 * ctx->M));
  return configure(ctx, centers, axes, n_contacts, contacts, false);
}

extern "C" int lcp_update_dev(lcp_ctx* ctx, const double* centers, const double* axes) {
  if (!ctx || !centers) return LCP_ERR_INVALID_ARG;
  return configure(ctx, centers, axes, 0, nullptr, true);
}

// Forward Euler step of Eq. (dvi): U = U_nc + M D x; c += dt U; Janus axis
// rotated by the angle |Omega| dt about Omega (Rodrigues' formula).
__global__ void k_advance(int M, double dt, const double* __restrict__ c, const double* __restrict__ e,
                          const double* __restrict__ unc, const double* __restrict__ mdx, int has_axes,
                          double* __restrict__ cn, double* __restrict__ en) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M) return;
  double u[6];
  for (int k = 0; k < 6; k++) u[k] = unc[6 * i + k] + mdx[6 * i + k];
  for (int d = 0; d < 3; d++) cn[3 * i + d] = c[3 * i + d] + dt * u[d];
  if (!has_axes) return;
  const double wx = u[3], wy = u[4], wz = u[5];
  const double wn = sqrt(wx * wx + wy * wy + wz * wz);
  double ex = e[3 * i], ey = e[3 * i + 1], ez = e[3 * i + 2];
  if (wn > 0.0) {
    const double th = wn * dt, kx = wx / wn, ky = wy / wn, kz = wz / wn;
    const double ct = cos(th), st = sin(th), kd = kx * ex + ky * ey + kz * ez;
    const double cx = ky * ez - kz * ey, cy = kz * ex - kx * ez, cz = kx * ey - ky * ex;
    const double nx = ex * ct + cx * st + kx * kd * (1.0 - ct);
    const double ny = ey * ct + cy * st + ky * kd * (1.0 - ct);
    const double nz = ez * ct + cz * st + kz * kd * (1.0 - ct);
    const double nn = sqrt(nx * nx + ny * ny + nz * nz);
    ex = nx / nn;
    ey = ny / nn;
    ez = nz / nn;
  }
  en[3 * i] = ex;
  en[3 * i + 1] = ey;
  en[3 * i + 2] = ez;
}

extern "C" int lcp_step(lcp_ctx* ctx, double dt, double* centers_out, double* axes_out) {
  if (!ctx || !(dt > 0.0)) return LCP_ERR_INVALID_ARG;
  if (!ctx->have_solution) { ctx->err = "lcp_step needs a solved LCP (call lcp_solve first)"; return LCP_ERR_INVALID_ARG; }
  const int M = ctx->M;
  // the solution and its body pairs, carried onto the next step's contacts below
  const bool carry = (ctx->cfg.warm_start & LCP_WARM_FORCES) && ctx->x_prev && ctx->n > 0;
  const int n_prev = carry ? ctx->n : 0;
  if (carry) {
    LCP_CUDA(cudaMemcpyAsync(ctx->x_prev, ctx->pq_outer.x, sizeof(double) * n_prev, cudaMemcpyDeviceToDevice,
                             ctx->stream));
    LCP_CUDA(cudaMemcpyAsync(ctx->ci_prev, ctx->ci, sizeof(int) * n_prev, cudaMemcpyDeviceToDevice, ctx->stream));
    LCP_CUDA(cudaMemcpyAsync(ctx->cj_prev, ctx->cj, sizeof(int) * n_prev, cudaMemcpyDeviceToDevice, ctx->stream));
  }
  ++ctx->nlaunch, k_advance<<<(M + 127) / 128, 128, 0, ctx->stream>>>(M, dt, ctx->centers, ctx->axes, ctx->U_nc,
                                                                     ctx->MDx, ctx->has_axes, ctx->cnext, ctx->anext);
  LCP_CUDA(cudaGetLastError());
  LCP_TRY(configure(ctx, ctx->cnext, ctx->has_axes ? ctx->anext : nullptr, 0, nullptr, true, true));
  ctx->have_solution = false;
  if (carry) {
    LCP_TRY(contacts_carry(ctx, n_prev));
    ctx->x_warm_valid = ctx->n > 0;
  }
  if (centers_out) LCP_TRY(copy_out(ctx, centers_out, ctx->centers, 3 * (size_t)M));
  if (axes_out && ctx->has_axes) LCP_TRY(copy_out(ctx, axes_out, ctx->axes, 3 * (size_t)M));
  return LCP_OK;
}

// Kernel timing: CUDA events around every stresslet-sum launch while enabled.
extern "C" int lcp_profile(lcp_ctx* ctx, int enable) {
  if (!ctx) return LCP_ERR_INVALID_ARG;
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
  ctx->ev_pool.clear();
  ctx->ev_kind.clear();
  for (int k = 0; k < 8; k++) {
    ctx->prof_ms[k] = 0.0;
    ctx->prof_n[k] = 0;
  }
  ctx->timed_key = -1;
  ctx->prof = enable != 0;
  return LCP_OK;
}

// Device bytes a context of this size will hold (same buffers as lcp_setup,
// with n_contacts contacts), for admission decisions before creating it.
extern "C" int lcp_footprint_estimate(const lcp_config* cfg, int n_bodies, int n_contacts, size_t* bytes) {
  if (!cfg || !bytes || n_bodies < 1 || n_contacts < 0) return LCP_ERR_INVALID_ARG;
  const size_t M = n_bodies, ns = (size_t)cfg->n_theta * cfg->n_phi, N = M * ns, L = 3 * N;
  const size_t m = cfg->gmres_restart, R = cfg->memory, K = cfg->kmax;
  const size_t n = n_contacts > 64 ? n_contacts : 64;
  const size_t pairs = M * (M - 1) / 2 > 0 ? M * (M - 1) / 2 : 1;
  size_t b = 0;
  b += sizeof(double) * L * (m + 1) + (cfg->precondition ? sizeof(double) * L * m : 0);   // Krylov bases
  b += sizeof(double) * L * 6 + sizeof(float) * L * 3;                                      // node vectors
  if (cfg->warm_start & LCP_WARM_FORCES)                                                    // carried forces
    b += (sizeof(double) * 2 + sizeof(int) * 2) * pairs;
  if (cfg->recycle > 0)                                                                      // reuse pairs
    b += sizeof(double) * (L * (2 * (size_t)cfg->recycle + 2) + 3 * (size_t)cfg->recycle);
  const size_t ntb = (N + 511) / 512, units = ntb * M / 2 + 1;                               // symmetric pair sum
  const size_t slots = std::min(units, 2 + M / std::max<size_t>(1, units / 304));
  b += sizeof(double) * L * std::max<size_t>(6, slots) + stokes_sym_bytes(n_bodies, (int)ns); // partial slots
  b += sizeof(double) * ((m + 1) * m + 6 * m + 16 + (m + 2) * 304);                          // Hessenberg, dots
  b += sizeof(double) * (8 * ns + 36) + sizeof(float) * 6 * ns + sizeof(double) * 30 * M + sizeof(float) * 8 * M;
  b += (sizeof(int) * 2 + sizeof(double) * 4) * pairs + sizeof(int) * M * (M + 2);           // contact buffers
  if (cfg->self_quadrature)                                                                  // self correction
    b += (sizeof(float) + sizeof(double)) * 9 * ns * ns + (cfg->precondition ? 0 : sizeof(float) * 4 * L);
  if (cfg->precondition)                                                                     // preconditioner
    b += sizeof(double) * 9 * ns * ns * 3 + sizeof(float) * 9 * ns * ns + sizeof(float) * 4 * L;
  b += sizeof(double) * n * (6 + 2 * K) + sizeof(int) * (2 * n + 1);                         // arena
  b += 2 * sizeof(double) * (n * (8 + 6 * R) + 3 * R * R + 64);                              // PQN states
  *bytes = b + (b >> 4);                                                                     // 1/16 slack
  if (cfg->lowfi_n_theta > 0) {   // the coarse-grid context
    lcp_config lc = *cfg;
    lc.n_theta = cfg->lowfi_n_theta;
    lc.n_phi = cfg->lowfi_n_phi;
    lc.memory = 1;
    lc.lowfi_n_theta = 0;
    size_t lb = 0;
    lcp_footprint_estimate(&lc, n_bodies, 0, &lb);
    *bytes += lb;
  }
  return LCP_OK;
}

extern "C" int lcp_footprint(const lcp_ctx* ctx, size_t* bytes) {
  if (!ctx || !bytes) return LCP_ERR_INVALID_ARG;
  *bytes = ctx->bytes + (ctx->lo ? ctx->lo->bytes : 0);
  return LCP_OK;
}

extern "C" const char* lcp_kernel_variant(const lcp_ctx* ctx) { return ctx ? stokes_variant_name(ctx) : ""; }

extern "C" int lcp_select_kernel_variant(lcp_ctx* ctx, const char* name) {
  if (!ctx || !name) return LCP_ERR_INVALID_ARG;
  return stokes_select_variant(ctx, name);
}

extern "C" int lcp_launch_count(const lcp_ctx* ctx, unsigned long long* count) {
  if (!ctx || !count) return LCP_ERR_INVALID_ARG;
  *count = ctx->nlaunch;
  return LCP_OK;
}

extern "C" int lcp_solve_counters(const lcp_ctx* ctx, int fidelity, long long* solves, long long* gmres_iterations,
                                   long long* recycled) {
  if (!ctx || !solves || !gmres_iterations || !recycled) return LCP_ERR_INVALID_ARG;
  const lcp_ctx* c = ctx;
  if (fidelity == LCP_LOW_BIE) {
    if (!ctx->lo) return LCP_ERR_INVALID_ARG;
    c = ctx->lo;
  } else if (fidelity != LCP_HIGH) {
    return LCP_ERR_INVALID_ARG;
  }
  *solves = c->tot_solves;
  *gmres_iterations = c->tot_gmres;
  *recycled = c->tot_recycled;
  return LCP_OK;
}

extern "C" int lcp_profile_read(lcp_ctx* ctx, int kind, int* count, double* total_ms) {
  if (!ctx || !count || !total_ms) return LCP_ERR_INVALID_ARG;
  LCP_CUDA(cudaStreamSynchronize(ctx->stream));
  int c = 0;
  double t = 0.0;
  if (kind >= 0 && kind < 8) {   // launches inside timed graph replays
    c = ctx->prof_n[kind];
    t = ctx->prof_ms[kind];
  }
  for (size_t k = 0; k < ctx->ev_kind.size(); k++) {
    if (ctx->ev_kind[k] != kind) continue;
    float ms = 0.f;
    LCP_CUDA(cudaEventElapsedTime(&ms, ctx->ev_pool[2 * k], ctx->ev_pool[2 * k + 1]));
    c++;
    t += ms;
  }
  *count = c;
  *total_ms = t;
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
  cudaGetDevice(&ctx->device);
  if (cfg->own_stream) {
    if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      g_setup_error = "could not create the context's stream";
      delete ctx;
      return LCP_ERR_CUDA;
    }
    ctx->owns_stream = true;
  }
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
  if (ctx->lo) lcp_destroy(ctx->lo);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  else cudaDeviceSynchronize();
  for (auto& g : ctx->agraphs) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    for (cudaEvent_t e : g.ev) cudaEventDestroy(e);
  }
  for (void* p : ctx->allocs) cudaFree(p);
  if (ctx->arena) cudaFree(ctx->arena);
  for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
  if (ctx->hscal) cudaFreeHost(ctx->hscal);
  if (ctx->owns_stream) cudaStreamDestroy(ctx->stream);
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
  if (include_slip && !ctx->has_axes) { ctx->err = "no Janus axes were given at set-up"; return LCP_ERR_INVALID_ARG; }
  if (fidelity == LCP_HIGH) {
    return mobility_solve(ctx, FT, include_slip, UO);
  } else if (fidelity == LCP_LOW_RPY) {
    if (include_slip) { ctx->err = "the RPY operator has no slip term"; return LCP_ERR_INVALID_ARG; }
    return rpy_apply(ctx, FT, UO);
  } else if (fidelity == LCP_LOW_BIE) {
    if (include_slip) { ctx->err = "the low-fidelity grid has no slip term"; return LCP_ERR_INVALID_ARG; }
    if (!ctx->lo) { ctx->err = "no low-fidelity grid configured (lowfi_n_theta = 0)"; return LCP_ERR_INVALID_ARG; }
    const int st = mobility_solve(ctx->lo, FT, 0, UO);
    if (st != LCP_OK) ctx->err = "low-fidelity grid: " + ctx->lo->err;
    return st;
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
    LCP_TRY(mvp_rpy(ctx, ctx->tmp_n2, ctx->tmp_n3));
  } else if (fidelity == LCP_LOW_BIE) {
    LCP_TRY(mvp_lowbie(ctx, ctx->tmp_n2, ctx->tmp_n3));
  } else {
    ctx->err = "unknown fidelity";
    return LCP_ERR_INVALID_ARG;
  }
  return copy_out(ctx, Ax, ctx->tmp_n3, ctx->n);
}

extern "C" int lcp_solve_dev(lcp_ctx* ctx, int method, double tol, const double* x0, double* x, lcp_stats* st) {
  if (!ctx || (ctx->n && !x) || !(tol >= 0.0)) return LCP_ERR_INVALID_ARG;
  if (method != LCP_MONO_PQN && method != LCP_BI_PQN && method != LCP_BB_PGD) { ctx->err = "unknown method"; return LCP_ERR_INVALID_ARG; }
  return lcp_solve_device(ctx, method, tol, x0, x, st);
}

extern "C" int lcp_solve(lcp_ctx* ctx, int method, double tol, const double* x0, double* x, lcp_stats* st) {
  if (!ctx || (ctx->n && !x) || !(tol >= 0.0)) return LCP_ERR_INVALID_ARG;
  if (method != LCP_MONO_PQN && method != LCP_BI_PQN && method != LCP_BB_PGD) { ctx->err = "unknown method"; return LCP_ERR_INVALID_ARG; }
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
  if (precision != LCP_FP64 && precision != LCP_MIXED && precision != LCP_DF64) return LCP_ERR_INVALID_ARG;
  LCP_TRY(stokes_apply(ctx, phi, out, precision));
  LCP_CUDA(cudaStreamSynchronize(ctx->stream));
  return LCP_OK;
}

extern "C" int lcp_stokes_rhs_dev(lcp_ctx* ctx, const double* FT, int include_slip, double* rhs) {
  if (!ctx || !FT || !rhs) return LCP_ERR_INVALID_ARG;
  if (include_slip && !ctx->has_axes) { ctx->err = "no Janus axes were given at set-up"; return LCP_ERR_INVALID_ARG; }
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
