// Geometry and contact set-up kernels (Sec. 3 of the paper: Eq. collisional-set
// and the contact matrix D; Sec. 5.1: order-p surface discretisation).
#include <cstdio>
#include <map>
#include <mutex>
#include <cstring>

#include "common.cuh"

// Gauss-Legendre nodes/weights by Newton's method on the three-term recurrence
// of the Legendre polynomials, then the product sphere rule.  One block.
// tmpl64[q] = {xi(3), wn(3), w, 0} with wn = -(3 / 4 pi) w n, n = xi / a.
__global__ void k_template(int nt, int np, double a, double* tmpl64, float* tmpl32,
                           double* tnodes) {
  const int ns = nt * np;
  if (threadIdx.x < nt) {
    const int i = threadIdx.x;
    double t = cos(LCP_PI * (i + 0.75) / (nt + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; it++) {
      double p0 = 1.0, p1 = t;
      for (int k = 1; k < nt; k++) {
        double p2 = ((2 * k + 1) * t * p1 - k * p0) / (k + 1);
        p0 = p1;
        p1 = p2;
      }
      dp = nt * (t * p1 - p0) / (t * t - 1.0);
      double dt = p1 / dp;
      t -= dt;
      if (fabs(dt) < 1e-16) break;
    }
    {
      double p0 = 1.0, p1 = t;
      for (int k = 1; k < nt; k++) {
        double p2 = ((2 * k + 1) * t * p1 - k * p0) / (k + 1);
        p0 = p1;
        p1 = p2;
      }
      dp = nt * (t * p1 - p0) / (t * t - 1.0);
    }
    const int j = nt - 1 - i;            // ascending order of t
    tnodes[2 * j] = t;
    tnodes[2 * j + 1] = 2.0 / ((1.0 - t * t) * dp * dp);
  }
  __syncthreads();
  const double c = -3.0 / (4.0 * LCP_PI);
  for (int q = threadIdx.x; q < ns; q += blockDim.x) {
    const int j = q / np, k = q % np;
    const double t = tnodes[2 * j], wt = tnodes[2 * j + 1];
    const double st = sqrt(1.0 - t * t);
    const double ph = 2.0 * LCP_PI * k / np;
    const double nx = st * cos(ph), ny = st * sin(ph), nz = t;
    const double w = a * a * wt * 2.0 * LCP_PI / np;
    double* o = tmpl64 + 8 * q;
    o[0] = a * nx; o[1] = a * ny; o[2] = a * nz;
    o[3] = c * w * nx; o[4] = c * w * ny; o[5] = c * w * nz;
    o[6] = w; o[7] = 0.0;
    for (int d = 0; d < 6; d++) tmpl32[d * ns + q] = (float)o[d];
  }
}

__device__ void rigid_mode_dev(int k, const double* xi, double* out) {
  out[0] = out[1] = out[2] = 0.0;
  if (k < 3) { out[k] = 1.0; return; }
  const int e = k - 3;
  // e_e x xi
  const double ex = e == 0, ey = e == 1, ez = e == 2;
  out[0] = ey * xi[2] - ez * xi[1];
  out[1] = ez * xi[0] - ex * xi[2];
  out[2] = ex * xi[1] - ey * xi[0];
}

// 6x6 Gram matrix of the rigid modes under the quadrature weights, inverted
// by Gauss-Jordan elimination with partial pivoting.  One thread.
__global__ void k_gram_inverse(int ns, const double* tmpl64, double* ginv) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double G[6][12];
  for (int k = 0; k < 6; k++)
    for (int l = 0; l < 12; l++) G[k][l] = (l - 6 == k) ? 1.0 : 0.0;
  for (int q = 0; q < ns; q++) {
    const double* o = tmpl64 + 8 * q;
    double psi[6][3];
    for (int k = 0; k < 6; k++) rigid_mode_dev(k, o, psi[k]);
    for (int k = 0; k < 6; k++)
      for (int l = 0; l < 6; l++)
        G[k][l] += o[6] * (psi[k][0] * psi[l][0] + psi[k][1] * psi[l][1] + psi[k][2] * psi[l][2]);
  }
  for (int k = 0; k < 6; k++) {
    int piv = k;
    for (int i = k + 1; i < 6; i++) if (fabs(G[i][k]) > fabs(G[piv][k])) piv = i;
    for (int l = 0; l < 12; l++) { double t = G[k][l]; G[k][l] = G[piv][l]; G[piv][l] = t; }
    const double inv = 1.0 / G[k][k];
    for (int l = 0; l < 12; l++) G[k][l] *= inv;
    for (int i = 0; i < 6; i++) {
      if (i == k) continue;
      const double f = G[i][k];
      for (int l = 0; l < 12; l++) G[i][l] -= f * G[k][l];
    }
  }
  for (int k = 0; k < 6; k++)
    for (int l = 0; l < 6; l++) ginv[6 * k + l] = G[k][6 + l];
}

// Centres split into float hi + lo parts for the FP32 pair kernel.
__global__ void k_centers32(int M, const double* c, float* c32) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M) return;
  for (int d = 0; d < 3; d++) {
    const float hi = __double2float_rn(c[3 * i + d]);
    const float lo = __double2float_rn(c[3 * i + d] - (double)hi);
    c32[8 * i + d] = hi;
    c32[8 * i + 4 + d] = lo;
  }
  c32[8 * i + 3] = 0.f;
  c32[8 * i + 7] = 0.f;
}

// Eq. (collisional-set): flag every pair i < j with gap <= delta.
__global__ void k_pair_flags(int M, const double* c, double rc, double delta, int* flags) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= M * M) return;
  const int i = t / M, j = t % M;
  int f = 0;
  if (i < j) {
    const double dx = c[3 * j] - c[3 * i], dy = c[3 * j + 1] - c[3 * i + 1], dz = c[3 * j + 2] - c[3 * i + 2];
    const double r = sqrt(dx * dx + dy * dy + dz * dz);
    f = (r - 2.0 * rc) <= delta;
  }
  flags[t] = f;
}

// Exclusive scan of the flags in one block (lexicographic pair order), then
// compaction of the contacts: normal (c_j - c_i)/|c_j - c_i|, gap.
__global__ void k_compact_pairs(int M, const double* c, double rc, const int* flags, int* count,
                                int cap, int* ci, int* cj, double* cnrm, double* gap) {
  __shared__ int base;
  __shared__ int warp_tot[32];
  const int total = M * M;
  if (threadIdx.x == 0) base = 0;
  __syncthreads();
  for (int start = 0; start < total; start += blockDim.x) {
    const int t = start + threadIdx.x;
    const int f = t < total ? flags[t] : 0;
    // block exclusive scan
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int v = f;
    for (int o = 1; o < 32; o <<= 1) {
      int u = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += u;
    }
    if (lane == 31) warp_tot[wid] = v;
    __syncthreads();
    if (wid == 0) {
      int w = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : 0;
      for (int o = 1; o < 32; o <<= 1) {
        int u = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += u;
      }
      warp_tot[lane] = w;
    }
    __syncthreads();
    const int excl = base + (wid > 0 ? warp_tot[wid - 1] : 0) + v - f;
    if (f && excl < cap) {
      const int i = t / M, j = t % M;
      const double dx = c[3 * j] - c[3 * i], dy = c[3 * j + 1] - c[3 * i + 1], dz = c[3 * j + 2] - c[3 * i + 2];
      const double r = sqrt(dx * dx + dy * dy + dz * dz);
      ci[excl] = i;
      cj[excl] = j;
      cnrm[3 * excl] = dx / r;
      cnrm[3 * excl + 1] = dy / r;
      cnrm[3 * excl + 2] = dz / r;
      gap[excl] = r - 2.0 * rc;
    }
    __syncthreads();
    if (threadIdx.x == 0) base += warp_tot[(blockDim.x >> 5) - 1];
    __syncthreads();
  }
  if (threadIdx.x == 0) *count = base;
}

// Body -> contact lists (CSR), contacts of a body in increasing order.
// bc_idx entry = 2 l + 1 when the body is the second body j of contact l
// (force +n), 2 l when it is the first body i (force -n).
__global__ void k_body_csr_count(int M, int n, const int* ci, const int* cj, int* cnt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M) return;
  int c = 0;
  for (int l = 0; l < n; l++) c += (ci[l] == i) + (cj[l] == i);
  cnt[i] = c;
}
__global__ void k_body_csr_fill(int M, int n, const int* ci, const int* cj, const int* ptr, int* idx) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M) return;
  int o = ptr[i];
  for (int l = 0; l < n; l++) {
    if (ci[l] == i) idx[o++] = 2 * l;
    if (cj[l] == i) idx[o++] = 2 * l + 1;
  }
}
__global__ void k_scan_small(int M, const int* cnt, int* ptr) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int s = 0;
  for (int i = 0; i < M; i++) { ptr[i] = s; s += cnt[i]; }
  ptr[M] = s;
}

cudaError_t raise_smem_limit(const void* kernel, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, size_t> limits;
  int dev = 0;
  const cudaError_t ed = cudaGetDevice(&dev);
  if (ed != cudaSuccess) return ed;
  std::lock_guard<std::mutex> lock(mu);
  size_t& cur = limits[std::make_pair(dev, kernel)];
  if (bytes <= cur) return cudaSuccess;
  const cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) cur = bytes;
  return e;
}

void* ctx_alloc(lcp_ctx* ctx, size_t bytes) {
  void* p = nullptr;
  if (bytes == 0) bytes = 16;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    ctx->err = "cudaMalloc of " + std::to_string(bytes) + " bytes failed";
    return nullptr;
  }
  ctx->allocs.push_back(p);
  ctx->bytes += bytes;
  return p;
}

// Template, Gram inverse and the fixed-size contact buffers (once per context).
int geometry_build(lcp_ctx* ctx) {
  const int ns = ctx->ns, M = ctx->M;
  ctx->tmpl64 = (double*)ctx_alloc(ctx, sizeof(double) * 8 * ns);
  ctx->tmpl32 = (float*)ctx_alloc(ctx, sizeof(float) * 6 * ns);
  ctx->ginv = (double*)ctx_alloc(ctx, sizeof(double) * 36);
  double* tn = (double*)ctx_alloc(ctx, sizeof(double) * 2 * ctx->cfg.n_theta);
  ctx->centers32 = (float*)ctx_alloc(ctx, sizeof(float) * 8 * M);
  ctx->pair_cap = M * (M - 1) / 2 > 0 ? M * (M - 1) / 2 : 1;
  const int cap = ctx->pair_cap;
  ctx->flags = (int*)ctx_alloc(ctx, sizeof(int) * (size_t)M * M);
  ctx->csr_cnt = (int*)ctx_alloc(ctx, sizeof(int) * M);
  ctx->bc_ptr = (int*)ctx_alloc(ctx, sizeof(int) * (M + 1));
  ctx->ci = (int*)ctx_alloc(ctx, sizeof(int) * cap);
  ctx->cj = (int*)ctx_alloc(ctx, sizeof(int) * cap);
  ctx->cnrm = (double*)ctx_alloc(ctx, sizeof(double) * 3 * cap);
  ctx->gap = (double*)ctx_alloc(ctx, sizeof(double) * cap);
  if (!ctx->tmpl64 || !ctx->tmpl32 || !ctx->ginv || !tn || !ctx->centers32 || !ctx->flags || !ctx->csr_cnt ||
      !ctx->bc_ptr || !ctx->ci || !ctx->cj || !ctx->cnrm || !ctx->gap)
    return LCP_ERR_OOM;
  if (ctx->cfg.warm_start & LCP_WARM_FORCES) {
    ctx->x_prev = (double*)ctx_alloc(ctx, sizeof(double) * cap);
    ctx->x_warm = (double*)ctx_alloc(ctx, sizeof(double) * cap);
    ctx->ci_prev = (int*)ctx_alloc(ctx, sizeof(int) * cap);
    ctx->cj_prev = (int*)ctx_alloc(ctx, sizeof(int) * cap);
    if (!ctx->x_prev || !ctx->x_warm || !ctx->ci_prev || !ctx->cj_prev) return LCP_ERR_OOM;
  }
  ++ctx->nlaunch, k_template<<<1, 256, 0, ctx->stream>>>(ctx->cfg.n_theta, ctx->cfg.n_phi, ctx->cfg.radius, ctx->tmpl64,
                                         ctx->tmpl32, tn);
  ++ctx->nlaunch, k_gram_inverse<<<1, 32, 0, ctx->stream>>>(ns, ctx->tmpl64, ctx->ginv);
  LCP_CUDA(cudaGetLastError());
  return LCP_OK;
}

// hi/lo split of the (new) centres.
int geometry_update(lcp_ctx* ctx) {
  ++ctx->nlaunch, k_centers32<<<(ctx->M + 127) / 128, 128, 0, ctx->stream>>>(ctx->M, ctx->centers, ctx->centers32);
  LCP_CUDA(cudaGetLastError());
  return LCP_OK;
}

int contacts_detect(lcp_ctx* ctx, int* n_out) {
  const int M = ctx->M;
  int* cnt = (int*)(ctx->dscal + 63);
  ++ctx->nlaunch, k_pair_flags<<<(M * M + 255) / 256, 256, 0, ctx->stream>>>(M, ctx->centers, ctx->cfg.contact_radius,
                                                               ctx->cfg.delta, ctx->flags);
  ++ctx->nlaunch, k_compact_pairs<<<1, 1024, 0, ctx->stream>>>(M, ctx->centers, ctx->cfg.contact_radius, ctx->flags, cnt,
                                              ctx->pair_cap, ctx->ci, ctx->cj, ctx->cnrm, ctx->gap);
  LCP_CUDA(cudaGetLastError());
  LCP_CUDA(cudaMemcpyAsync(ctx->hscal + 63, cnt, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  LCP_CUDA(cudaStreamSynchronize(ctx->stream));
  int n = 0;
  memcpy(&n, ctx->hscal + 63, sizeof(int));
  *n_out = n;
  return LCP_OK;
}

// x_warm[l] = the previous step's force on the same body pair (i, j), or 0 for
// a new contact.  Linear search: the previous list need not be sorted (caller
// contacts), and n_prev is a few hundred to a few thousand.
__global__ void k_carry_forces(int n, const int* __restrict__ ci, const int* __restrict__ cj, int n_prev,
                               const int* __restrict__ pi, const int* __restrict__ pj,
                               const double* __restrict__ x_prev, double* __restrict__ x_warm) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= n) return;
  const int i = ci[l], j = cj[l];
  double v = 0.0;
  for (int k = 0; k < n_prev; k++)
    if (pi[k] == i && pj[k] == j) {
      v = x_prev[k];
      break;
    }
  x_warm[l] = v;
}

int contacts_carry(lcp_ctx* ctx, int n_prev) {
  if (ctx->n == 0) return LCP_OK;
  ++ctx->nlaunch, k_carry_forces<<<(ctx->n + 127) / 128, 128, 0, ctx->stream>>>(
                      ctx->n, ctx->ci, ctx->cj, n_prev, ctx->ci_prev, ctx->cj_prev, ctx->x_prev, ctx->x_warm);
  LCP_CUDA(cudaGetLastError());
  return LCP_OK;
}

int contacts_upload(lcp_ctx* ctx, int n, const lcp_contact* c) {
  if (n > ctx->pair_cap) {
    ctx->err = "more contacts than body pairs";
    return LCP_ERR_INVALID_ARG;
  }
  std::vector<int> hi(n), hj(n);
  std::vector<double> hn(3 * (size_t)n), hg(n);
  for (int l = 0; l < n; l++) {
    if (c[l].i < 0 || c[l].j < 0 || c[l].i >= ctx->M || c[l].j >= ctx->M || c[l].i == c[l].j) {
      ctx->err = "contact " + std::to_string(l) + " names an invalid body pair";
      return LCP_ERR_INVALID_ARG;
    }
    hi[l] = c[l].i;
    hj[l] = c[l].j;
    for (int d = 0; d < 3; d++) hn[3 * l + d] = c[l].normal[d];
    hg[l] = c[l].gap;
  }
  if (n > 0) {
    LCP_CUDA(cudaMemcpyAsync(ctx->ci, hi.data(), sizeof(int) * n, cudaMemcpyHostToDevice, ctx->stream));
    LCP_CUDA(cudaMemcpyAsync(ctx->cj, hj.data(), sizeof(int) * n, cudaMemcpyHostToDevice, ctx->stream));
    LCP_CUDA(cudaMemcpyAsync(ctx->cnrm, hn.data(), sizeof(double) * 3 * n, cudaMemcpyHostToDevice, ctx->stream));
    LCP_CUDA(cudaMemcpyAsync(ctx->gap, hg.data(), sizeof(double) * n, cudaMemcpyHostToDevice, ctx->stream));
    LCP_CUDA(cudaStreamSynchronize(ctx->stream));
  }
  return LCP_OK;
}

// bc_idx must hold 2 n entries (contact arena).
int contacts_csr(lcp_ctx* ctx) {
  const int M = ctx->M, n = ctx->n;
  ++ctx->nlaunch, k_body_csr_count<<<(M + 127) / 128, 128, 0, ctx->stream>>>(M, n, ctx->ci, ctx->cj, ctx->csr_cnt);
  ++ctx->nlaunch, k_scan_small<<<1, 32, 0, ctx->stream>>>(M, ctx->csr_cnt, ctx->bc_ptr);
  ++ctx->nlaunch, k_body_csr_fill<<<(M + 127) / 128, 128, 0, ctx->stream>>>(M, n, ctx->ci, ctx->cj, ctx->bc_ptr, ctx->bc_idx);
  LCP_CUDA(cudaGetLastError());
  return LCP_OK;
}
