// Mobility solves: restarted GMRES with FP64 Arnoldi (classical Gram-Schmidt
// applied twice) on (K + P) phi = rhs, in FP64 or as GMRES iterative
// refinement with FP32 stresslet sums (the paper fixes GMRES with tolerance
// eps_gmres for its traction BIE, Sec. 5.1 and Sec. 6); the contact matrix D
// and its transpose (Sec. 3); and the Rotne-Prager-Yamakawa low-fidelity
// mobility.
#include <cmath>

#include "common.cuh"

int stokes_velocity(lcp_ctx* ctx, const double* phi, double* UO);

namespace {
constexpr int DOT_THREADS = 256;
}

// Fused Gram-Schmidt pass over one chunk of rows per block:
//   w -= sum_{k < nu} h[k] V[k]            (skipped when nu = 0), then
//   out[k] = Vd[k] . w  for k < nd          (Vd may be w itself: the norm).
// Block b owns rows [b c, (b+1) c), so the update and the partial dots of its
// rows need no grid-wide barrier; partial dots are reduced warp-per-vector,
// written to partial[k * G + b], and the last block to finish adds them in
// block order (deterministic).
__global__ void __launch_bounds__(DOT_THREADS)
k_update_dots(int L, int nu, const double* __restrict__ V, size_t ldv, const double* __restrict__ h, double* w,
              int nd, const double* Vd, size_t ldvd, double* __restrict__ partial, double* __restrict__ out,
              unsigned int* __restrict__ counter) {
  __shared__ bool last;
  const int G = gridDim.x;
  const int chunk = (L + G - 1) / G;
  const int i0 = blockIdx.x * chunk, i1 = min(L, i0 + chunk);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  if (nu > 0) {
    for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
      double s = w[i];
      for (int k = 0; k < nu; k++) s -= h[k] * V[(size_t)k * ldv + i];
      w[i] = s;
    }
    __syncthreads();
  }
  for (int k = warp; k < nd; k += nwarps) {
    const double* v = Vd + (size_t)k * ldvd;
    double s = 0.0;
    for (int i = i0 + lane; i < i1; i += 32) s += v[i] * w[i];
    s = warp_sum(s);
    if (lane == 0) partial[(size_t)k * G + blockIdx.x] = s;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(counter, 1u) == (unsigned)(G - 1));
  __syncthreads();
  if (!last) return;
  __threadfence();
  for (int k = warp; k < nd; k += nwarps) {
    double s = 0.0;
    for (int b = lane; b < G; b += 32) s += ((volatile double*)partial)[(size_t)k * G + b];
    s = warp_sum(s);
    if (lane == 0) out[k] = s;
  }
  if (threadIdx.x == 0) *counter = 0u;
}

// y = a * x (+ y if accumulate)
__global__ void k_scale(int L, const double* __restrict__ x, const double* __restrict__ a, double* __restrict__ y,
                        int invert, int accumulate) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= L) return;
  const double s = invert ? 1.0 / a[0] : a[0];
  y[i] = accumulate ? y[i] + s * x[i] : s * x[i];
}

__global__ void k_sub(int L, const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ c) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < L) c[i] = a[i] - b[i];
}
__global__ void k_add(int L, const double* __restrict__ a, double* __restrict__ c) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < L) c[i] += a[i];
}
// y = s x
__global__ void k_scale_into(int L, double s, const double* __restrict__ x, double* __restrict__ y) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < L) y[i] = s * x[i];
}

// GMRES bookkeeping on the device (one thread).  Work layout (doubles):
// H[(m+1) * m] column j at H + j * (m+1); cs[m]; sn[m]; g[m+1]; y[m];
// h1[m+1]; h2[m+1]; hn[1]; inv[1]; beta[1].
struct GW {
  double *H, *cs, *sn, *g, *y, *h1, *h2, *hn, *beta;
};
__device__ GW gw_map(double* base, int m) {
  GW w;
  w.H = base;
  w.cs = w.H + (size_t)(m + 1) * m;
  w.sn = w.cs + m;
  w.g = w.sn + m;
  w.y = w.g + (m + 1);
  w.h1 = w.y + m;
  w.h2 = w.h1 + (m + 1);
  w.hn = w.h2 + (m + 1);
  w.beta = w.hn + 1;
  return w;
}

// Start of a cycle: beta = sqrt(hn); g = (beta, 0, ...); status[0] = beta.
__global__ void k_gmres_start(double* base, int m, double* status) {
  GW w = gw_map(base, m);
  const double beta = sqrt(w.hn[0]);
  w.beta[0] = beta;
  for (int k = 0; k <= m; k++) w.g[k] = 0.0;
  w.g[0] = beta;
  status[0] = beta;
}

// Column j of H from the two Gram-Schmidt passes, Givens rotations, new
// residual estimate |g[j+1]| into status[0]; hn becomes 1/H[j+1][j].
__global__ void k_gmres_column(double* base, int m, int j, double* status) {
  GW w = gw_map(base, m);
  double* Hj = w.H + (size_t)j * (m + 1);
  for (int k = 0; k <= j; k++) Hj[k] = w.h1[k] + w.h2[k];
  const double hnext = sqrt(w.hn[0]);
  Hj[j + 1] = hnext;
  for (int k = 0; k < j; k++) {
    const double a = Hj[k], b = Hj[k + 1];
    Hj[k] = w.cs[k] * a + w.sn[k] * b;
    Hj[k + 1] = -w.sn[k] * a + w.cs[k] * b;
  }
  const double a = Hj[j], b = Hj[j + 1];
  const double r = sqrt(a * a + b * b);
  w.cs[j] = a / r;
  w.sn[j] = b / r;
  Hj[j] = r;
  Hj[j + 1] = 0.0;
  w.g[j + 1] = -w.sn[j] * w.g[j];
  w.g[j] = w.cs[j] * w.g[j];
  w.hn[0] = hnext > 0.0 ? 1.0 / hnext : 0.0;
  status[0] = fabs(w.g[j + 1]);
  status[1] = hnext;
}

// Back substitution H y = g for the first k columns.
__global__ void k_gmres_solve(double* base, int m, int k) {
  GW w = gw_map(base, m);
  for (int r = k - 1; r >= 0; r--) {
    double s = w.g[r];
    for (int c = r + 1; c < k; c++) s -= w.H[(size_t)c * (m + 1) + r] * w.y[c];
    w.y[r] = s / w.H[(size_t)r * (m + 1) + r];
  }
}

// phi += sum_k y[k] V[k]
__global__ void k_gmres_update(int L, int k, const double* __restrict__ V, size_t ldv, const double* __restrict__ y,
                               double* __restrict__ phi) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= L) return;
  double s = phi[i];
  for (int c = 0; c < k; c++) s += y[c] * V[(size_t)c * ldv + i];
  phi[i] = s;
}

// ----------------------------------------------------------- D and D^T
// F_i = sum over contacts l of body i of (-n_l or +n_l) x_l; torques 0 (spheres).
__global__ void k_scatter(int M, const int* __restrict__ ptr, const int* __restrict__ idx,
                          const double* __restrict__ cnrm, const double* __restrict__ x, double* __restrict__ FT) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M) return;
  double f0 = 0.0, f1 = 0.0, f2 = 0.0;
  for (int e = ptr[i]; e < ptr[i + 1]; e++) {
    const int code = idx[e];
    const int l = code >> 1;
    const double s = (code & 1) ? x[l] : -x[l];
    f0 += s * cnrm[3 * l];
    f1 += s * cnrm[3 * l + 1];
    f2 += s * cnrm[3 * l + 2];
  }
  double* o = FT + 6 * i;
  o[0] = f0; o[1] = f1; o[2] = f2; o[3] = 0.0; o[4] = 0.0; o[5] = 0.0;
}

// (D^T U)_l = n_l . (U_j - U_i) (+ add_l)
__global__ void k_gather(int n, const int* __restrict__ ci, const int* __restrict__ cj,
                         const double* __restrict__ cnrm, const double* __restrict__ UO,
                         const double* __restrict__ add, double* __restrict__ out) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= n) return;
  const double* ui = UO + 6 * ci[l];
  const double* uj = UO + 6 * cj[l];
  double v = cnrm[3 * l] * (uj[0] - ui[0]) + cnrm[3 * l + 1] * (uj[1] - ui[1]) + cnrm[3 * l + 2] * (uj[2] - ui[2]);
  if (add) v += add[l];
  out[l] = v;
}

// ----------------------------------------------------------- RPY
// One warp per target body; lanes stride over source bodies; fixed reduction.
__global__ void k_rpy(int M, double a, double mu, const double* __restrict__ c, const double* __restrict__ FT,
                      double* __restrict__ UO) {
  const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= M) return;
  double u[6] = {0, 0, 0, 0, 0, 0};
  const double k8 = 1.0 / (8.0 * LCP_PI * mu);
  for (int j = lane; j < M; j += 32) {
    const double* f = FT + 6 * j;
    if (j == i) {
      const double st = 1.0 / (6.0 * LCP_PI * mu * a), sr = 1.0 / (8.0 * LCP_PI * mu * a * a * a);
      for (int d = 0; d < 3; d++) { u[d] += st * f[d]; u[3 + d] += sr * f[3 + d]; }
      continue;
    }
    const double rx = c[3 * i] - c[3 * j], ry = c[3 * i + 1] - c[3 * j + 1], rz = c[3 * i + 2] - c[3 * j + 2];
    const double r = sqrt(rx * rx + ry * ry + rz * rz);
    const double hx = rx / r, hy = ry / r, hz = rz / r;
    const double a2r2 = a * a / (r * r);
    const double ct = k8 / r * (1.0 + 2.0 * a2r2 / 3.0), cp = k8 / r * (1.0 - 2.0 * a2r2);
    const double hF = hx * f[0] + hy * f[1] + hz * f[2];
    u[0] += ct * f[0] + cp * hF * hx;
    u[1] += ct * f[1] + cp * hF * hy;
    u[2] += ct * f[2] + cp * hF * hz;
    const double r3 = k8 / (r * r * r);
    // U_i += (T_j x r) / (8 pi mu r^3) ; Omega_i += (F_j x r) / (8 pi mu r^3)
    u[0] += r3 * (f[4] * rz - f[5] * ry);
    u[1] += r3 * (f[5] * rx - f[3] * rz);
    u[2] += r3 * (f[3] * ry - f[4] * rx);
    u[3] += r3 * (f[1] * rz - f[2] * ry);
    u[4] += r3 * (f[2] * rx - f[0] * rz);
    u[5] += r3 * (f[0] * ry - f[1] * rx);
    // Omega_i += (3 h h^T - I) T_j / (16 pi mu r^3)
    const double hT = hx * f[3] + hy * f[4] + hz * f[5];
    const double rr = 0.5 * r3;
    u[3] += rr * (3.0 * hT * hx - f[3]);
    u[4] += rr * (3.0 * hT * hy - f[4]);
    u[5] += rr * (3.0 * hT * hz - f[5]);
  }
#pragma unroll
  for (int d = 0; d < 6; d++) u[d] = warp_sum(u[d]);
  if (lane == 0)
    for (int d = 0; d < 6; d++) UO[6 * i + d] = u[d];
}

// ------------------------------------------------------------------ host side
static int blocks_for(int L, int t) { return (L + t - 1) / t; }

static int update_dots(lcp_ctx* ctx, int L, int nu, const double* V, size_t ldv, const double* h, double* w,
                       int nd, const double* Vd, size_t ldvd, double* out) {
  ++ctx->nlaunch, k_update_dots<<<ctx->dot_blocks, DOT_THREADS, 0, ctx->stream>>>(
                      L, nu, V, ldv, h, w, nd, Vd, ldvd, ctx->dotp, out, (unsigned int*)(ctx->dscal + 60));
  LCP_CUDA(cudaGetLastError());
  return LCP_OK;
}

static int dots(lcp_ctx* ctx, int L, int nv, const double* V, size_t ldv, const double* w, double* out) {
  return update_dots(ctx, L, 0, nullptr, 0, nullptr, const_cast<double*>(w), nv, V, ldv, out);
}

static int read_status(lcp_ctx* ctx, double* vals, int count) {
  LCP_CUDA(cudaMemcpyAsync(ctx->hscal, ctx->dscal, sizeof(double) * count, cudaMemcpyDeviceToHost, ctx->stream));
  LCP_CUDA(cudaStreamSynchronize(ctx->stream));
  for (int k = 0; k < count; k++) vals[k] = ctx->hscal[k];
  return LCP_OK;
}

// Arnoldi step j of GMRES: z_j = Minv v_j (flexible right preconditioning),
// w = (K + P) z_j, classical Gram-Schmidt twice (each update fused with the
// next dots), the Givens column of H, v_{j+1} = w / H[j+1][j], and the copy of
// the residual estimate and H[j+1][j] to the pinned host mirror.
static int arnoldi_step(lcp_ctx* ctx, int j, int prec) {
  const int L = 3 * ctx->N, m = ctx->m, T = 256;
  const size_t ldv = (size_t)L;
  double* base = ctx->H;
  const size_t oH = 0, ocs = oH + (size_t)(m + 1) * m, osn = ocs + m, og = osn + m, oy = og + (m + 1),
               oh1 = oy + m, oh2 = oh1 + (m + 1), ohn = oh2 + (m + 1);
  double* h1 = base + oh1;
  double* h2 = base + oh2;
  double* hn = base + ohn;
  double* vj = ctx->V + (size_t)j * ldv;
  double* vn = ctx->V + (size_t)(j + 1) * ldv;
  if (ctx->Z) {
    double* zj = ctx->Z + (size_t)j * ldv;
    LCP_TRY(precond_apply(ctx, vj, zj));
    vj = zj;
  }
  LCP_TRY(stokes_apply(ctx, vj, vn, prec));
  LCP_TRY(dots(ctx, L, j + 1, ctx->V, ldv, vn, h1));
  LCP_TRY(update_dots(ctx, L, j + 1, ctx->V, ldv, h1, vn, j + 1, ctx->V, ldv, h2));
  LCP_TRY(update_dots(ctx, L, j + 1, ctx->V, ldv, h2, vn, 1, vn, ldv, hn));
  ++ctx->nlaunch, k_gmres_column<<<1, 1, 0, ctx->stream>>>(base, m, j, ctx->dscal);
  ++ctx->nlaunch, k_scale<<<blocks_for(L, T), T, 0, ctx->stream>>>(L, vn, hn, vn, 0, 0);
  LCP_CUDA(cudaMemcpyAsync(ctx->hscal, ctx->dscal, sizeof(double) * 2, cudaMemcpyDeviceToHost, ctx->stream));
  LCP_CUDA(cudaGetLastError());
  return LCP_OK;
}

// Launches Arnoldi step j as a captured CUDA graph (one per column, operator
// precision and kernel timing on or off, captured on first use and replayed
// by every later solve of the context), or directly when the context runs on
// the legacy default stream (not capturable).  With kernel timing on, the
// graph records its own event pairs around the pair-sum launch; the caller
// reads them with arnoldi_timing after synchronising.
static int arnoldi_launch(lcp_ctx* ctx, int j, int prec) {
  if (!ctx->stream) return arnoldi_step(ctx, j, prec);
  const int key = (j * 3 + prec) * 2 + (ctx->prof ? 1 : 0);
  const int stamp = ctx->sym ? 1000 + ctx->sym_v : ctx->v32;
  if ((int)ctx->agraphs.size() <= key) ctx->agraphs.resize(key + 1);
  lcp_ctx::ArnoldiGraph& g = ctx->agraphs[key];
  if (!g.exec || g.stamp != stamp) {
    if (g.exec) {
      LCP_CUDA(cudaStreamSynchronize(ctx->stream));
      cudaGraphExecDestroy(g.exec);
      g.exec = nullptr;
    }
    for (cudaEvent_t e : g.ev) cudaEventDestroy(e);
    g.ev.clear();
    g.ev_kind.clear();
    const unsigned long long n0 = ctx->nlaunch;
    const int c32 = ctx->c_fp32, c64 = ctx->c_fp64, cdf = ctx->c_df64;
    LCP_CUDA(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
    if (ctx->prof) {
      ctx->cap_ev = &g.ev;
      ctx->cap_kind = &g.ev_kind;
    }
    const int st = arnoldi_step(ctx, j, prec);
    ctx->cap_ev = nullptr;
    ctx->cap_kind = nullptr;
    cudaGraph_t graph = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(ctx->stream, &graph);
    if (st != LCP_OK || ce != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      if (st != LCP_OK) return st;
      ctx->err = std::string("GMRES graph capture: ") + cudaGetErrorString(ce);
      return LCP_ERR_CUDA;
    }
    const cudaError_t ie = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) {
      g.exec = nullptr;
      ctx->err = std::string("GMRES graph instantiation: ") + cudaGetErrorString(ie);
      return LCP_ERR_CUDA;
    }
    g.kernels = ctx->nlaunch - n0;
    g.c32 = ctx->c_fp32 - c32;
    g.c64 = ctx->c_fp64 - c64;
    g.cdf = ctx->c_df64 - cdf;
    ctx->nlaunch = n0;   // nothing ran during the capture
    ctx->c_fp32 = c32;
    ctx->c_fp64 = c64;
    ctx->c_df64 = cdf;
    g.stamp = stamp;
  }
  LCP_CUDA(cudaGraphLaunch(g.exec, ctx->stream));
  ctx->nlaunch += g.kernels;
  ctx->c_fp32 += g.c32;
  ctx->c_fp64 += g.c64;
  ctx->c_df64 += g.cdf;
  ctx->timed_key = g.ev.empty() ? -1 : key;
  return LCP_OK;
}

// After the stream has synchronised: adds the kernel times the last timed
// graph replay recorded (before that graph can run, and record, again).
static int arnoldi_timing(lcp_ctx* ctx) {
  if (ctx->timed_key < 0) return LCP_OK;
  const lcp_ctx::ArnoldiGraph& g = ctx->agraphs[ctx->timed_key];
  ctx->timed_key = -1;
  for (size_t k = 0; k < g.ev_kind.size(); k++) {
    float ms = 0.f;
    LCP_CUDA(cudaEventElapsedTime(&ms, g.ev[2 * k], g.ev[2 * k + 1]));
    const int kind = g.ev_kind[k];
    if (kind >= 0 && kind < 8) {
      ctx->prof_ms[kind] += ms;
      ctx->prof_n[kind]++;
    }
  }
  return LCP_OK;
}

// Restarted GMRES(m) on (K + P) phi = rhs with operator precision `prec`;
// flexible GMRES (Saad 1993) with the block-diagonal preconditioner when it
// is enabled: the solution is assembled from the stored preconditioned
// vectors, so the preconditioner's precision does not limit the accuracy.
// phi holds the initial guess (zero_init: assume phi = 0 and skip the first
// residual apply).  Stops when the residual estimate <= tol_abs or after
// maxit iterations.  Returns the iterations used in *its, the last residual
// estimate in *res_out.
static int gmres(lcp_ctx* ctx, const double* rhs, double* phi, int zero_init, double tol_abs, int prec,
                 int maxit, int* its, double* res_out) {
  const int L = 3 * ctx->N, m = ctx->m;
  const size_t ldv = (size_t)L;
  double* base = ctx->H;
  // offsets of the scalar slots inside the work array (host mirror of gw_map)
  const size_t oH = 0, ocs = oH + (size_t)(m + 1) * m, osn = ocs + m, og = osn + m, oy = og + (m + 1),
               oh1 = oy + m, oh2 = oh1 + (m + 1), ohn = oh2 + (m + 1);
  double* hn = base + ohn;
  double* y = base + oy;
  int total = 0;
  double res = 0.0;
  bool first = true;
  const int T = 256;
  for (;;) {
    // r = rhs - A phi into V[0]
    if (first && zero_init) {
      LCP_CUDA(cudaMemcpyAsync(ctx->V, rhs, sizeof(double) * L, cudaMemcpyDeviceToDevice, ctx->stream));
    } else {
      LCP_TRY(stokes_apply(ctx, phi, ctx->wv, prec));
      ++ctx->nlaunch, k_sub<<<blocks_for(L, T), T, 0, ctx->stream>>>(L, rhs, ctx->wv, ctx->V);
    }
    first = false;
    LCP_TRY(dots(ctx, L, 1, ctx->V, ldv, ctx->V, hn));
    ++ctx->nlaunch, k_gmres_start<<<1, 1, 0, ctx->stream>>>(base, m, ctx->dscal);
    double st[2];
    LCP_TRY(read_status(ctx, st, 1));
    res = st[0];
    if (!(res == res)) { ctx->err = "GMRES: NaN residual"; return LCP_ERR_NUMERICAL; }
    if (res <= tol_abs || total >= maxit) break;
    ++ctx->nlaunch, k_scale<<<blocks_for(L, T), T, 0, ctx->stream>>>(L, ctx->V, base + ohn + 1, ctx->V, 1, 0);  // V0 /= beta
    int j = 0;
    for (; j < m; j++) {
      LCP_TRY(arnoldi_launch(ctx, j, prec));
      total++;
      LCP_CUDA(cudaStreamSynchronize(ctx->stream));
      LCP_TRY(arnoldi_timing(ctx));
      st[0] = ctx->hscal[0];
      st[1] = ctx->hscal[1];
      res = st[0];
      if (!(res == res)) { ctx->err = "GMRES: NaN residual"; return LCP_ERR_NUMERICAL; }
      if (res <= tol_abs || total >= maxit || st[1] == 0.0) { j++; break; }
    }
    ++ctx->nlaunch, k_gmres_solve<<<1, 1, 0, ctx->stream>>>(base, m, j);
    ++ctx->nlaunch, k_gmres_update<<<blocks_for(L, T), T, 0, ctx->stream>>>(L, j, ctx->Z ? ctx->Z : ctx->V, ldv,
                                                                             y, phi);
    LCP_CUDA(cudaGetLastError());
    if (res <= tol_abs || total >= maxit) break;
  }
  *its = total;
  *res_out = res;
  return LCP_OK;
}

static int norm2(lcp_ctx* ctx, const double* v, int L, double* out) {
  double* slot = ctx->dscal + 8;
  LCP_TRY(dots(ctx, L, 1, v, (size_t)L, v, slot));
  LCP_CUDA(cudaMemcpyAsync(ctx->hscal + 8, slot, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  LCP_CUDA(cudaStreamSynchronize(ctx->stream));
  *out = std::sqrt(ctx->hscal[8]);
  return LCP_OK;
}

// --------------------------------------------------- reuse across solves
// The mobility solves of one configuration share the operator K + P, and the
// right-hand sides of the successive MVPs of one LCP differ little.  The
// context keeps up to rc_max pairs (psi_k, w_k) from its earlier solves, with
// w_k ~= (K + P) psi_k and the w_k orthonormal.  A solve may start from the
// Galerkin projection phi0 = Psi c, c = W^T rhs, whose residual is predicted
// as rhs - W c (Fischer's projection method for successive right-hand
// sides).  After each solve its pair enters: the direction the solve moved
// (phi - phi_start) and its image (start residual - final residual),
// orthogonalised against the kept w_k by classical Gram-Schmidt applied twice
// (the same coefficients applied to the psi_k) and normalised.  Once every
// slot is in use the set restarts from the newest solve alone: its whole
// solution and right-hand side (less the final residual) as the one pair.
// The w_k only choose the start: each solve's accepted residual is computed
// from its own iterate, so an inexact image costs iterations, not accuracy.

// A projected start is taken when it predicts a residual below
// RC_USE ||rhs||: at least one decade, worth more than the one operator
// application that the FP64 and FP32-only solves spend on its exact residual.
static constexpr double RC_USE = 0.1;

// c = a - c
__global__ void k_from_sub(int L, const double* __restrict__ a, double* __restrict__ c) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < L) c[i] = a[i] - c[i];
}
// c = c - b
__global__ void k_sub_from(int L, const double* __restrict__ b, double* __restrict__ c) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < L) c[i] -= b[i];
}

void recycle_reset(lcp_ctx* ctx) {
  ctx->rc_count = 0;
  if (ctx->lo) recycle_reset(ctx->lo);
}

// c = W^T rhs (into rc_h), phi = Psi c, r = rhs - W c; *rn = ||r||.
static int recycle_project(lcp_ctx* ctx, const double* rhs, double* phi, double* r, double* rn) {
  const int L = 3 * ctx->N, m = ctx->rc_count, T = 256;
  const size_t ld = (size_t)L;
  double* c = ctx->rc_h;
  LCP_TRY(dots(ctx, L, m, ctx->rc_w, ld, rhs, c));
  LCP_CUDA(cudaMemsetAsync(phi, 0, sizeof(double) * L, ctx->stream));
  ++ctx->nlaunch, k_gmres_update<<<blocks_for(L, T), T, 0, ctx->stream>>>(L, m, ctx->rc_psi, ld, c, phi);
  LCP_CUDA(cudaGetLastError());
  LCP_CUDA(cudaMemcpyAsync(r, rhs, sizeof(double) * L, cudaMemcpyDeviceToDevice, ctx->stream));
  LCP_TRY(update_dots(ctx, L, m, ctx->rc_w, ld, c, r, 1, r, ld, ctx->dscal + 8));   // r -= W c; ||r||^2
  LCP_CUDA(cudaMemcpyAsync(ctx->hscal + 8, ctx->dscal + 8, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  LCP_CUDA(cudaStreamSynchronize(ctx->stream));
  *rn = std::sqrt(ctx->hscal[8]);
  return LCP_OK;
}

// Enters the pair (rc_phi0, rc_r0) = (direction, image) of the solve just
// finished into the free slot rc_count (< rc_max); skipped when its
// orthogonalised image is not above wmin (no new direction).
static int recycle_add(lcp_ctx* ctx, double wmin) {
  const int L = 3 * ctx->N, m = ctx->rc_count, T = 256;
  const size_t ld = (size_t)L;
  double* p = ctx->rc_phi0;
  double* w = ctx->rc_r0;
  double* h1 = ctx->rc_h + ctx->rc_max;
  double* h2 = ctx->rc_h + 2 * ctx->rc_max;
  if (m > 0) {
    LCP_TRY(dots(ctx, L, m, ctx->rc_w, ld, w, h1));
    LCP_TRY(update_dots(ctx, L, m, ctx->rc_w, ld, h1, w, m, ctx->rc_w, ld, h2));
    LCP_TRY(update_dots(ctx, L, m, ctx->rc_w, ld, h2, w, 0, nullptr, 0, nullptr));
    LCP_TRY(update_dots(ctx, L, m, ctx->rc_psi, ld, h1, p, 0, nullptr, 0, nullptr));
    LCP_TRY(update_dots(ctx, L, m, ctx->rc_psi, ld, h2, p, 0, nullptr, 0, nullptr));
  }
  double wn = 0.0;
  LCP_TRY(norm2(ctx, w, L, &wn));
  if (!(wn > wmin) || !std::isfinite(wn)) return LCP_OK;
  ++ctx->nlaunch, k_scale_into<<<blocks_for(L, T), T, 0, ctx->stream>>>(L, 1.0 / wn, w, ctx->rc_w + m * ld);
  ++ctx->nlaunch, k_scale_into<<<blocks_for(L, T), T, 0, ctx->stream>>>(L, 1.0 / wn, p, ctx->rc_psi + m * ld);
  LCP_CUDA(cudaGetLastError());
  ctx->rc_count++;
  return LCP_OK;
}

// Solve (K + P) phi = rhs to ||rhs - (K + P) phi|| <= gmres_tol ||rhs||.
// FP64: GMRES on the FP64 operator.  MIXED: iterative refinement.  Each sweep
// solves for a correction d with GMRES on the FP32 operator (FP64 Arnoldi) to
// inner_tol relative.  The residual after the first sweep is recomputed with
// the high-accuracy operator (FP64 or double-FP32 sums, residual_precision);
// later residuals are updated, r <- r - (K + P)_32 d, which is accurate to
// ~eps32 ||K|| ||d|| because those corrections are small (the FP32
// operator's relative error eps32 is ~4e-7).  A correction larger than
// IR_UPDATE_MAX ||phi|| falls back to a high-accuracy residual.  The
// low-fidelity grid (fp32_only) runs GMRES on the FP32 operator alone.
static constexpr double IR_UPDATE_MAX = 1e-5;

// phi0 (or NULL): initial guess (the previous slip density along a
// trajectory); its residual is taken with the solve's accurate operator, so
// the guess only has to be close, not exact.  Without phi0 the start is the
// projection on the kept pairs when it predicts a residual below
// RC_USE ||rhs||, else zero.
int density_solve(lcp_ctx* ctx, const double* rhs, double* phi, const double* phi0) {
  const int L = 3 * ctx->N;
  const int T = 256;
  double bn = 0.0;
  LCP_TRY(norm2(ctx, rhs, L, &bn));
  if (bn == 0.0) {
    LCP_CUDA(cudaMemsetAsync(phi, 0, sizeof(double) * L, ctx->stream));
    return LCP_OK;
  }
  const double tol = ctx->cfg.gmres_tol * bn;
  const bool keep = ctx->rc_max > 0;
  const bool refine = ctx->cfg.precision != LCP_FP64 && !ctx->fp32_only;
  // start: 0 zero, 1 phi0, 2 projection (predicted residual in ctx->res, norm rn)
  int start = 0;
  double rn = bn;
  if (phi0) {
    LCP_CUDA(cudaMemcpyAsync(phi, phi0, sizeof(double) * L, cudaMemcpyDeviceToDevice, ctx->stream));
    start = 1;
  } else if (keep && ctx->rc_count > 0) {
    double rp = 0.0;
    LCP_TRY(recycle_project(ctx, rhs, phi, ctx->res, &rp));
    if (rp <= RC_USE * bn) {
      start = 2;
      rn = rp;
      ctx->c_recycled++;
    }
  }
  if (start == 0) LCP_CUDA(cudaMemsetAsync(phi, 0, sizeof(double) * L, ctx->stream));
  int its = 0;
  double res = 0.0;
  if (!refine) {
    const int prec = ctx->cfg.precision == LCP_FP64 ? LCP_FP64 : LCP_MIXED;
    double* r0 = keep ? ctx->rc_r0 : ctx->res;
    double* d = keep ? ctx->rc_phi0 : ctx->dphi;
    if (start == 0) {
      LCP_TRY(gmres(ctx, rhs, phi, 1, tol, prec, ctx->cfg.gmres_maxit, &its, &res));
      if (keep && its > 0) {
        LCP_CUDA(cudaMemcpyAsync(d, phi, sizeof(double) * L, cudaMemcpyDeviceToDevice, ctx->stream));
        LCP_CUDA(cudaMemcpyAsync(r0, rhs, sizeof(double) * L, cudaMemcpyDeviceToDevice, ctx->stream));
      }
    } else {
      // exact start residual with the solve's operator, then the correction
      LCP_TRY(stokes_apply(ctx, phi, ctx->wv, prec));
      ++ctx->nlaunch, k_sub<<<blocks_for(L, T), T, 0, ctx->stream>>>(L, rhs, ctx->wv, r0);
      LCP_CUDA(cudaMemsetAsync(d, 0, sizeof(double) * L, ctx->stream));
      LCP_TRY(gmres(ctx, r0, d, 1, tol, prec, ctx->cfg.gmres_maxit, &its, &res));
      ++ctx->nlaunch, k_add<<<blocks_for(L, T), T, 0, ctx->stream>>>(L, d, phi);
      LCP_CUDA(cudaGetLastError());
    }
    ctx->c_gmres += its;
    if (res > tol) {
      ctx->err = "GMRES did not reach its tolerance";
      return LCP_ERR_NOT_CONVERGED;
    }
    // the image of the direction is r0 up to the final residual (<= tol)
    if (keep && its > 0) {
      if (ctx->rc_count == ctx->rc_max) {   // full: restart from this solve
        ctx->rc_count = 0;
        LCP_CUDA(cudaMemcpyAsync(d, phi, sizeof(double) * L, cudaMemcpyDeviceToDevice, ctx->stream));
        LCP_CUDA(cudaMemcpyAsync(r0, rhs, sizeof(double) * L, cudaMemcpyDeviceToDevice, ctx->stream));
      }
      LCP_TRY(recycle_add(ctx, tol));
    }
    return LCP_OK;
  }
  // mixed precision: refinement from the start's residual
  if (start == 1) {
    LCP_TRY(stokes_apply(ctx, phi, ctx->wv, ctx->cfg.residual_precision));
    ++ctx->nlaunch, k_sub<<<blocks_for(L, T), T, 0, ctx->stream>>>(L, rhs, ctx->wv, ctx->res);
    LCP_TRY(norm2(ctx, ctx->res, L, &rn));
    if (!(rn == rn)) { ctx->err = "refinement: NaN residual"; return LCP_ERR_NUMERICAL; }
    if (rn <= tol) return LCP_OK;
  } else if (start == 0) {
    LCP_CUDA(cudaMemcpyAsync(ctx->res, rhs, sizeof(double) * L, cudaMemcpyDeviceToDevice, ctx->stream));
  }
  if (keep) {
    LCP_CUDA(cudaMemcpyAsync(ctx->rc_phi0, phi, sizeof(double) * L, cudaMemcpyDeviceToDevice, ctx->stream));
    LCP_CUDA(cudaMemcpyAsync(ctx->rc_r0, ctx->res, sizeof(double) * L, cudaMemcpyDeviceToDevice, ctx->stream));
  }
  for (int sweep = 0; sweep < ctx->cfg.ir_maxit; sweep++) {
    LCP_CUDA(cudaMemsetAsync(ctx->dphi, 0, sizeof(double) * L, ctx->stream));
    const double tin = std::max(ctx->cfg.inner_tol * rn, 0.5 * tol);
    LCP_TRY(gmres(ctx, ctx->res, ctx->dphi, 1, tin, LCP_MIXED, ctx->cfg.gmres_maxit, &its, &res));
    ctx->c_gmres += its;
    ++ctx->nlaunch, k_add<<<blocks_for(L, T), T, 0, ctx->stream>>>(L, ctx->dphi, phi);
    double dn = 0.0, pn = 0.0;
    LCP_TRY(norm2(ctx, ctx->dphi, L, &dn));
    LCP_TRY(norm2(ctx, phi, L, &pn));
    // the first sweep always ends with an accurate residual: after a
    // projected start it replaces the predicted one
    if (sweep == 0 || dn > IR_UPDATE_MAX * pn) {
      LCP_TRY(stokes_apply(ctx, phi, ctx->wv, ctx->cfg.residual_precision));
      ++ctx->nlaunch, k_sub<<<blocks_for(L, T), T, 0, ctx->stream>>>(L, rhs, ctx->wv, ctx->res);
    } else {
      LCP_TRY(stokes_apply(ctx, ctx->dphi, ctx->wv, LCP_MIXED));
      ++ctx->nlaunch, k_sub<<<blocks_for(L, T), T, 0, ctx->stream>>>(L, ctx->res, ctx->wv, ctx->res);
    }
    LCP_TRY(norm2(ctx, ctx->res, L, &rn));
    if (!(rn == rn)) { ctx->err = "refinement: NaN residual"; return LCP_ERR_NUMERICAL; }
    if (rn <= tol) {
      if (keep) {
        if (ctx->rc_count == ctx->rc_max) {   // full: restart from phi, image rhs - r_final
          ctx->rc_count = 0;
          LCP_CUDA(cudaMemcpyAsync(ctx->rc_phi0, phi, sizeof(double) * L, cudaMemcpyDeviceToDevice, ctx->stream));
          ++ctx->nlaunch, k_sub<<<blocks_for(L, T), T, 0, ctx->stream>>>(L, rhs, ctx->res, ctx->rc_r0);
        } else {   // direction phi - phi_start, image r_start - r_final
          ++ctx->nlaunch, k_from_sub<<<blocks_for(L, T), T, 0, ctx->stream>>>(L, phi, ctx->rc_phi0);
          ++ctx->nlaunch, k_sub_from<<<blocks_for(L, T), T, 0, ctx->stream>>>(L, ctx->res, ctx->rc_r0);
        }
        LCP_CUDA(cudaGetLastError());
        LCP_TRY(recycle_add(ctx, tol));
      }
      return LCP_OK;
    }
  }
  ctx->err = "iterative refinement did not reach the GMRES tolerance";
  return LCP_ERR_NOT_CONVERGED;
}

int mobility_solve(lcp_ctx* ctx, const double* FT, int include_slip, double* UO, const double* phi0) {
  LCP_TRY(stokes_rhs(ctx, FT, include_slip, ctx->rhs));
  const int g0 = ctx->c_gmres, r0 = ctx->c_recycled;
  const int st = density_solve(ctx, ctx->rhs, ctx->phi, phi0);
  ctx->tot_solves++;
  ctx->tot_gmres += ctx->c_gmres - g0;
  ctx->tot_recycled += ctx->c_recycled - r0;
  LCP_TRY(st);
  return stokes_velocity(ctx, ctx->phi, UO);
}

int scatter_D(lcp_ctx* ctx, const double* x, double* FT) {
  ++ctx->nlaunch, k_scatter<<<blocks_for(ctx->M, 128), 128, 0, ctx->stream>>>(ctx->M, ctx->bc_ptr, ctx->bc_idx, ctx->cnrm, x, FT);
  LCP_CUDA(cudaGetLastError());
  return LCP_OK;
}

int gather_Dt(lcp_ctx* ctx, const double* UO, double* out, const double* add) {
  if (ctx->n == 0) return LCP_OK;
  ++ctx->nlaunch, k_gather<<<blocks_for(ctx->n, 128), 128, 0, ctx->stream>>>(ctx->n, ctx->ci, ctx->cj, ctx->cnrm, UO, add, out);
  LCP_CUDA(cudaGetLastError());
  return LCP_OK;
}

int rpy_apply(lcp_ctx* ctx, const double* FT, double* UO) {
  ++ctx->nlaunch, k_rpy<<<blocks_for(ctx->M * 32, 128), 128, 0, ctx->stream>>>(ctx->M, ctx->cfg.radius, ctx->cfg.viscosity,
                                                                 ctx->centers, FT, UO);
  LCP_CUDA(cudaGetLastError());
  return LCP_OK;
}

int mvp_high(lcp_ctx* ctx, const double* x, double* Ax) {
  LCP_TRY(scatter_D(ctx, x, ctx->FT));
  LCP_TRY(mobility_solve(ctx, ctx->FT, 0, ctx->UO));
  return gather_Dt(ctx, ctx->UO, Ax, nullptr);
}

int mvp_rpy(lcp_ctx* ctx, const double* x, double* Ax) {
  LCP_TRY(scatter_D(ctx, x, ctx->FT));
  LCP_TRY(rpy_apply(ctx, ctx->FT, ctx->UO));
  return gather_Dt(ctx, ctx->UO, Ax, nullptr);
}

// Low-fidelity MVP through the coarse-grid context: the same D and D^T, the
// boundary-integral mobility of the coarse grid (Sec. 5.1, coarseness of the
// discretisation as fidelity).
int mvp_lowbie(lcp_ctx* ctx, const double* x, double* Ax) {
  lcp_ctx* lo = ctx->lo;
  if (!lo) { ctx->err = "no low-fidelity grid configured (lowfi_n_theta = 0)"; return LCP_ERR_INVALID_ARG; }
  LCP_TRY(scatter_D(ctx, x, ctx->FT));
  const int st = mobility_solve(lo, ctx->FT, 0, lo->UO);
  if (st != LCP_OK) { ctx->err = "low-fidelity grid: " + lo->err; return st; }
  return gather_Dt(ctx, lo->UO, Ax, nullptr);
}

int mvp_low(lcp_ctx* ctx, const double* x, double* Ax) {
  return ctx->lo ? mvp_lowbie(ctx, x, Ax) : mvp_rpy(ctx, x, Ax);
}
