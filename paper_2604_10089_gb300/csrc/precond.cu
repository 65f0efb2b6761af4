// Block-diagonal preconditioner for the boundary-integral solve.
//
// Every sphere carries the same quadrature template, so the operator of an
// isolated sphere, K_iso + P_iso (3 ns x 3 ns), is the same for all bodies and
// is the diagonal block of K + P up to the coupling through the other bodies.
// Its inverse is computed once per context (FP64 Gauss-Jordan), stored in
// FP32, and applied to every body as one small GEMM.  GMRES uses it as a
// flexible (right) preconditioner, so its FP32 rounding changes only the
// convergence rate, never the accuracy of the solution.
#include "common.cuh"

// Dense K_iso + P_iso of one sphere (row-major, n = 3 ns), off-diagonal K
// blocks and the P part; the K diagonal blocks are added by k_iso_diag.
__global__ void k_iso_matrix(int ns, const double* __restrict__ tmpl64, const double* __restrict__ ginv,
                             double* __restrict__ A) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ns * ns) return;
  const int p = t / ns, q = t % ns;
  const int n = 3 * ns;
  const double* xp = tmpl64 + 8 * p;
  const double* xq = tmpl64 + 8 * q;
  double blk[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  if (p != q) {
    const double r[3] = {xp[0] - xq[0], xp[1] - xq[1], xp[2] - xq[2]};
    const double r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
    const double ir = rsqrt(r2);
    const double s = (r[0] * xq[3] + r[1] * xq[4] + r[2] * xq[5]) * ir * ir * ir * ir * ir;
    for (int a = 0; a < 3; a++)
      for (int b = 0; b < 3; b++) blk[a][b] = s * r[a] * r[b];
  }
  // P block: sum_kl psi_k(xi_p)_a Ginv_kl psi_l(xi_q)_b w_q
  double psp[6][3], psq[6][3];
  for (int k = 0; k < 6; k++) {
    for (int a = 0; a < 3; a++) { psp[k][a] = 0.0; psq[k][a] = 0.0; }
    if (k < 3) { psp[k][k] = 1.0; psq[k][k] = 1.0; }
  }
  for (int e = 0; e < 3; e++) {   // e_e x xi
    const double ex = e == 0, ey = e == 1, ez = e == 2;
    psp[3 + e][0] = ey * xp[2] - ez * xp[1]; psp[3 + e][1] = ez * xp[0] - ex * xp[2]; psp[3 + e][2] = ex * xp[1] - ey * xp[0];
    psq[3 + e][0] = ey * xq[2] - ez * xq[1]; psq[3 + e][1] = ez * xq[0] - ex * xq[2]; psq[3 + e][2] = ex * xq[1] - ey * xq[0];
  }
  const double wq = xq[6];
  for (int a = 0; a < 3; a++)
    for (int b = 0; b < 3; b++) {
      double s = 0.0;
      for (int k = 0; k < 6; k++)
        for (int l = 0; l < 6; l++) s += psp[k][a] * ginv[6 * k + l] * psq[l][b];
      blk[a][b] += s * wq;
    }
  for (int a = 0; a < 3; a++)
    for (int b = 0; b < 3; b++) A[(size_t)(3 * p + a) * n + 3 * q + b] = blk[a][b];
}

// K diagonal blocks: -sum_{q != p} w_q T(xi_p - xi_q, n_q), one thread per p.
__global__ void k_iso_diag(int ns, const double* __restrict__ tmpl64, double* __restrict__ A) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= ns) return;
  const int n = 3 * ns;
  const double* xp = tmpl64 + 8 * p;
  double blk[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  for (int q = 0; q < ns; q++) {
    if (q == p) continue;
    const double* xq = tmpl64 + 8 * q;
    const double r[3] = {xp[0] - xq[0], xp[1] - xq[1], xp[2] - xq[2]};
    const double r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
    const double ir = rsqrt(r2);
    const double s = (r[0] * xq[3] + r[1] * xq[4] + r[2] * xq[5]) * ir * ir * ir * ir * ir;
    for (int a = 0; a < 3; a++)
      for (int b = 0; b < 3; b++) blk[a][b] += s * r[a] * r[b];
  }
  for (int a = 0; a < 3; a++)
    for (int b = 0; b < 3; b++) A[(size_t)(3 * p + a) * n + 3 * p + b] -= blk[a][b];
}

// Gauss-Jordan on the augmented [A | I] (n x 2n, row-major), pivot step k:
// one block finds the pivot row, swaps it into row k, scales row k and saves
// column k for the elimination.
__global__ void k_gj_step_pivot(int n, int k, double* __restrict__ Aug, double* __restrict__ colk) {
  __shared__ double bv[256];
  __shared__ int bi[256];
  const int w = 2 * n;
  double best = -1.0;
  int arg = k;
  for (int i = k + threadIdx.x; i < n; i += blockDim.x) {
    const double v = fabs(Aug[(size_t)i * w + k]);
    if (v > best || (v == best && i < arg)) { best = v; arg = i; }
  }
  bv[threadIdx.x] = best;
  bi[threadIdx.x] = arg;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      const double v = bv[threadIdx.x + s];
      const int i = bi[threadIdx.x + s];
      if (v > bv[threadIdx.x] || (v == bv[threadIdx.x] && i < bi[threadIdx.x])) { bv[threadIdx.x] = v; bi[threadIdx.x] = i; }
    }
    __syncthreads();
  }
  const int piv = bi[0];
  if (piv != k)
    for (int j = threadIdx.x; j < w; j += blockDim.x) {
      const double t = Aug[(size_t)k * w + j];
      Aug[(size_t)k * w + j] = Aug[(size_t)piv * w + j];
      Aug[(size_t)piv * w + j] = t;
    }
  __syncthreads();
  const double inv = 1.0 / Aug[(size_t)k * w + k];
  __syncthreads();
  for (int j = threadIdx.x; j < w; j += blockDim.x) Aug[(size_t)k * w + j] *= inv;
  for (int i = threadIdx.x; i < n; i += blockDim.x) colk[i] = (i == k) ? 0.0 : Aug[(size_t)i * w + k];
}

__global__ void k_gj_identity(int n, double* __restrict__ Aug) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) Aug[(size_t)i * 2 * n + n + i] = 1.0;
}

__global__ void k_gj_step_elim(int n, int k, double* __restrict__ Aug, const double* __restrict__ colk) {
  const int w = 2 * n;
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)n * w) return;
  const int i = (int)(t / w), j = (int)(t % w);
  if (i == k) return;
  Aug[t] -= colk[i] * Aug[(size_t)k * w + j];
}

__global__ void k_gj_extract(int n, const double* __restrict__ Aug, float* __restrict__ Minv) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)n * n) return;
  const int i = (int)(t / n), j = (int)(t % n);
  Minv[t] = (float)Aug[(size_t)i * 2 * n + n + j];
}

// z_b = Minv v_b for every body b: C (n x M) = Minv (n x n) B (n x M), B and C
// column-major with columns = bodies (the node-vector layout).  FP32 tiles,
// FP64 in.  The k range is split PT_KS ways so that the small GEMM fills the
// SMs with several CTAs each (one CTA per SM would wait on every tile load);
// split s writes its FP32 partial product to part[s][M][n] and k_precond_sum
// adds the splits in a fixed order.
constexpr int PT_R = 64, PT_C = 16, PT_K = 32, PT_KS = 4;
__global__ void __launch_bounds__(256) k_precond(int n, int M, int kc, const float* __restrict__ Minv,
                                                 const double* __restrict__ v, float* __restrict__ part) {
  __shared__ float As[PT_K][PT_R + 1];
  __shared__ float Bs[PT_C][PT_K + 1];
  const int r0 = blockIdx.x * PT_R, c0 = blockIdx.y * PT_C;
  const int ka = blockIdx.z * kc, kb = min(n, ka + kc);
  const int tr = threadIdx.x % PT_R;        // row within the tile
  const int tc = threadIdx.x / PT_R;        // 0..3: handles columns tc, tc+4, tc+8, tc+12
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  for (int k0 = ka; k0 < kb; k0 += PT_K) {
    for (int t = threadIdx.x; t < PT_R * PT_K; t += blockDim.x) {
      const int rr = t / PT_K, kk = t % PT_K;
      const int gr = r0 + rr, gk = k0 + kk;
      As[kk][rr] = (gr < n && gk < kb) ? Minv[(size_t)gr * n + gk] : 0.f;
    }
    for (int t = threadIdx.x; t < PT_C * PT_K; t += blockDim.x) {
      const int cc = t / PT_K, kk = t % PT_K;
      const int gc = c0 + cc, gk = k0 + kk;
      Bs[cc][kk] = (gc < M && gk < kb) ? (float)v[(size_t)gc * n + gk] : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < PT_K; kk++) {
      const float a = As[kk][tr];
#pragma unroll
      for (int u = 0; u < 4; u++) acc[u] = fmaf(a, Bs[tc + 4 * u][kk], acc[u]);
    }
    __syncthreads();
  }
  const int gr = r0 + tr;
  if (gr < n)
    for (int u = 0; u < 4; u++) {
      const int gc = c0 + tc + 4 * u;
      if (gc < M) part[((size_t)blockIdx.z * M + gc) * n + gr] = acc[u];
    }
}

// z = the sum of the splits (or z += it)
__global__ void k_precond_sum(int L, const float* __restrict__ part, double* __restrict__ z, int accumulate) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= L) return;
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < PT_KS; k++) s += (double)part[(size_t)k * L + i];
  z[i] = accumulate ? z[i] + s : s;
}

// A += Bt^T (n x n, row-major)
__global__ void k_add_transposed(int n, const double* __restrict__ Bt, double* __restrict__ A) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)n * n) return;
  const int i = (int)(t / n), j = (int)(t % n);
  A[t] += Bt[(size_t)j * n + i];
}

int precond_build(lcp_ctx* ctx) {
  const int ns = ctx->ns, n = 3 * ns;
  double* aug = (double*)ctx_alloc(ctx, sizeof(double) * (size_t)n * 2 * n);
  double* colk = (double*)ctx_alloc(ctx, sizeof(double) * n);
  ctx->pinv = (float*)ctx_alloc(ctx, sizeof(float) * (size_t)n * n);
  LCP_TRY(block_apply_reserve(ctx));
  if (!aug || !colk || !ctx->pinv) return LCP_ERR_OOM;
  // assemble K_iso + P_iso (n x n), then copy it into the left half of [A | I]
  double* tmp = (double*)ctx_alloc(ctx, sizeof(double) * (size_t)n * n);
  if (!tmp) return LCP_ERR_OOM;
  ++ctx->nlaunch, k_iso_matrix<<<(ns * ns + 127) / 128, 128, 0, ctx->stream>>>(ns, ctx->tmpl64, ctx->ginv, tmp);
  ++ctx->nlaunch, k_iso_diag<<<(ns + 127) / 128, 128, 0, ctx->stream>>>(ns, ctx->tmpl64, tmp);
  if (ctx->cself64t)   // the corrected self-interaction is part of the isolated sphere's operator
    ++ctx->nlaunch, k_add_transposed<<<(unsigned)(((size_t)n * n + 255) / 256), 256, 0, ctx->stream>>>(
                        n, ctx->cself64t, tmp);
  LCP_CUDA(cudaMemsetAsync(aug, 0, sizeof(double) * (size_t)n * 2 * n, ctx->stream));
  LCP_CUDA(cudaMemcpy2DAsync(aug, sizeof(double) * 2 * n, tmp, sizeof(double) * n, sizeof(double) * n, n,
                             cudaMemcpyDeviceToDevice, ctx->stream));
  ++ctx->nlaunch, k_gj_identity<<<(n + 127) / 128, 128, 0, ctx->stream>>>(n, aug);
  const size_t total = (size_t)n * 2 * n;
  for (int k = 0; k < n; k++) {
    ++ctx->nlaunch, k_gj_step_pivot<<<1, 256, 0, ctx->stream>>>(n, k, aug, colk);
    ++ctx->nlaunch, k_gj_step_elim<<<(unsigned)((total + 255) / 256), 256, 0, ctx->stream>>>(n, k, aug, colk);
  }
  ++ctx->nlaunch, k_gj_extract<<<(unsigned)(((size_t)n * n + 255) / 256), 256, 0, ctx->stream>>>(n, aug, ctx->pinv);
  LCP_CUDA(cudaGetLastError());
  LCP_CUDA(cudaStreamSynchronize(ctx->stream));
  return LCP_OK;
}

// The split-k partial products of the per-body block GEMMs (once per context).
int block_apply_reserve(lcp_ctx* ctx) {
  if (ctx->ppart) return LCP_OK;
  ctx->ppart = (float*)ctx_alloc(ctx, sizeof(float) * PT_KS * (size_t)3 * ctx->ns * ctx->M);
  return ctx->ppart ? LCP_OK : LCP_ERR_OOM;
}

// z_b = mat v_b (or z_b += mat v_b) for every body b; mat is 3 ns x 3 ns, FP32, row-major.
int block_apply32(lcp_ctx* ctx, const float* mat, const double* v, double* z, bool accumulate) {
  const int n = 3 * ctx->ns;
  const int kc = ((n + PT_K - 1) / PT_K + PT_KS - 1) / PT_KS * PT_K;
  dim3 grid((n + PT_R - 1) / PT_R, (ctx->M + PT_C - 1) / PT_C, PT_KS);
  ++ctx->nlaunch, k_precond<<<grid, 256, 0, ctx->stream>>>(n, ctx->M, kc, mat, v, ctx->ppart);
  const int L = n * ctx->M;
  ++ctx->nlaunch, k_precond_sum<<<(L + 255) / 256, 256, 0, ctx->stream>>>(L, ctx->ppart, z, accumulate ? 1 : 0);
  LCP_CUDA(cudaGetLastError());
  return LCP_OK;
}

int precond_apply(lcp_ctx* ctx, const double* v, double* z) {
  return block_apply32(ctx, ctx->pinv, v, z, false);
}
