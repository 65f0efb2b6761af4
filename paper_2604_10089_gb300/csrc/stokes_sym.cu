// Symmetric FP32 stresslet pair sum (the default inner-solve operator).
//
// For nodes p, q on different bodies, with r = x_p - x_q and d = phi_q - phi_p,
// the two ordered terms of (K phi) (Sec. 2, the double layer of the completed
// formulation),
//   target p, source q:  w_q T(r, n_q) d          = (r . wn_q) t r,
//   target q, source p:  w_p T(-r, n_p) (-d)      = (r . wn_p) t r,
// with wn = -(3/4pi) w n and t = (r . d) / |r|^5, share r, |r|^-5 and r . d.
// One evaluation therefore serves both targets: 15 instead of 23 FP32
// operations per ordered pair.  Pairs within one body are summed one way
// (forward only), as in the plain kernel.
//
// Work: target blocks of SYM_TB consecutive nodes (two per thread) times
// source bodies j >= the block's first body; a unit (tb, j) adds the forward
// terms of targets with body(p) <= j and the reverse terms of targets with
// body(p) < j.  Units are dealt in equal contiguous ranges to one wave of
// CTAs, as for the plain kernel.  Forward sums stay in registers along a row
// and go to partial[slot][p]; the reverse sums of unit (tb, j) are reduced
// over the CTA's 512 targets (a transposing warp reduction, then the 8 warps
// in order) and written to a per-unit row of `rev` (FP32), which the finish
// kernel adds in target-block order.  Everything is deterministic.
#include <vector>

#include "common.cuh"

namespace {

constexpr int SYM_THREADS = 256;
constexpr int SYM_TB = 2 * SYM_THREADS;   // targets per block
constexpr int SYM_WARPS = SYM_THREADS / 32;
constexpr int SYM_CHUNK = 8;               // source bodies staged per tile
constexpr float SYM_EPS = 1e-20f;          // r = 0 only for q = p: keeps |r|^-3 = 1e30 finite, the term 0

__device__ __forceinline__ float rsqrt_fast(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ void kahan(float& s, float& c, float v) {
  const float y = v - c;
  const float t = s + y;
  c = (t - s) - y;
  s = t;
}

struct SymUnits {
  int U, G, ntb, ns;
  const int* off;          // [ntb + 1]: first unit of each target block
  const long long* roff;   // [ntb]: first float of each target block's reverse rows
  __device__ __forceinline__ int start(int c) const { return (int)(((long long)c * U) / G); }
  __device__ __forceinline__ int cta_of(int u) const {
    int c = (int)(((long long)u * G) / U);
    while (c + 1 < G && start(c + 1) <= u) c++;
    while (c > 0 && start(c) > u) c--;
    return c;
  }
  __device__ __forceinline__ int first_body(int tb) const { return (int)(((long long)tb * SYM_TB) / ns); }
};

// One target (broadcast in e, nf, wp) against the source pair (q, q+1) held
// in the lanes of the float2 source values.
__device__ __forceinline__ void sym_pair(const float2 (&e)[3], const float2 (&nf)[3], const float2 (&wp)[3],
                                         float2 nx, float2 ny, float2 nz, float2 wx, float2 wy, float2 wz,
                                         float2 fx, float2 fy, float2 fz, float2 (&acc)[3], float2 (&rv)[3]) {
  const float2 rx = __fadd2_rn(e[0], nx);
  const float2 ry = __fadd2_rn(e[1], ny);
  const float2 rz = __fadd2_rn(e[2], nz);
  float2 r2 = __ffma2_rn(rx, rx, make_float2(SYM_EPS, SYM_EPS));
  r2 = __ffma2_rn(ry, ry, r2);
  r2 = __ffma2_rn(rz, rz, r2);
  const float2 ir = make_float2(rsqrt_fast(r2.x), rsqrt_fast(r2.y));
  const float2 i2 = __fmul2_rn(ir, ir);
  const float2 dx = __fadd2_rn(fx, nf[0]);
  const float2 dy = __fadd2_rn(fy, nf[1]);
  const float2 dz = __fadd2_rn(fz, nf[2]);
  float2 rd = __fmul2_rn(rx, dx);
  rd = __ffma2_rn(ry, dy, rd);
  rd = __ffma2_rn(rz, dz, rd);
  const float2 t = __fmul2_rn(__fmul2_rn(rd, i2), __fmul2_rn(i2, ir));
  float2 rq = __fmul2_rn(rx, wx);
  rq = __ffma2_rn(ry, wy, rq);
  rq = __ffma2_rn(rz, wz, rq);
  float2 rp = __fmul2_rn(rx, wp[0]);
  rp = __ffma2_rn(ry, wp[1], rp);
  rp = __ffma2_rn(rz, wp[2], rp);
  const float2 sf = __fmul2_rn(rq, t);
  const float2 sr = __fmul2_rn(rp, t);
  acc[0] = __ffma2_rn(sf, rx, acc[0]);
  acc[1] = __ffma2_rn(sf, ry, acc[1]);
  acc[2] = __ffma2_rn(sf, rz, acc[2]);
  rv[0] = __ffma2_rn(sr, rx, rv[0]);
  rv[1] = __ffma2_rn(sr, ry, rv[1]);
  rv[2] = __ffma2_rn(sr, rz, rv[2]);
}

// Sum 16 values over the 32 lanes of a warp with 16 shuffles: at each level
// a lane keeps half of its values and sends the other half to its partner.
// Afterwards lanes 2k and 2k+1 both hold the warp total of value k.
__device__ __forceinline__ float warp_transpose_sum16(float (&v)[16], int lane) {
  const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4, b1 = lane & 2;
  float w[8];
#pragma unroll
  for (int i = 0; i < 8; i++) {
    const float send = b4 ? v[i] : v[i + 8];
    const float keep = b4 ? v[i + 8] : v[i];
    w[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
  float x[4];
#pragma unroll
  for (int i = 0; i < 4; i++) {
    const float send = b3 ? w[i] : w[i + 4];
    const float keep = b3 ? w[i + 4] : w[i];
    x[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
  float y[2];
#pragma unroll
  for (int i = 0; i < 2; i++) {
    const float send = b2 ? x[i] : x[i + 2];
    const float keep = b2 ? x[i + 2] : x[i];
    y[i] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  }
  const float send = b1 ? y[0] : y[1];
  const float keep = b1 ? y[1] : y[0];
  float z = keep + __shfl_xor_sync(0xffffffffu, send, 2);
  z += __shfl_xor_sync(0xffffffffu, z, 1);
  return z;
}

}  // namespace

__global__ void __launch_bounds__(SYM_THREADS, 2)
k_pair32_sym(int N, int ns, int ns_pad, SymUnits su, const float* __restrict__ tmpl32, const float* __restrict__ c32,
             const float* __restrict__ phi32, double* __restrict__ partial, float* __restrict__ rev) {
  extern __shared__ float4 smem4[];
  float* sm = reinterpret_cast<float*>(smem4);
  float* s_nx = sm;                          // -xi per template node (padded)
  float* s_ny = s_nx + ns_pad;
  float* s_nz = s_ny + ns_pad;
  float* s_wx = s_nz + ns_pad;               // wn = -(3/4pi) w n
  float* s_wy = s_wx + ns_pad;
  float* s_wz = s_wy + ns_pad;
  float* s_f = s_wz + ns_pad;                // [3][SYM_CHUNK][ns_pad] staged source densities
  float* s_rev = s_f + 3 * SYM_CHUNK * ns_pad;   // [2][SYM_WARPS][3][ns_pad] per-warp reverse sums
  for (int q = threadIdx.x; q < ns_pad; q += blockDim.x) {
    const bool real = q < ns;
    s_nx[q] = real ? -tmpl32[q] : -1.0e3f;
    s_ny[q] = real ? -tmpl32[ns + q] : 0.f;
    s_nz[q] = real ? -tmpl32[2 * ns + q] : 0.f;
    s_wx[q] = real ? tmpl32[3 * ns + q] : 0.f;
    s_wy[q] = real ? tmpl32[4 * ns + q] : 0.f;
    s_wz[q] = real ? tmpl32[5 * ns + q] : 0.f;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c = blockIdx.x;
  int u = su.start(c);
  const int uend = su.start(c + 1);
  int buf = 0;
  while (u < uend) {
    int lo = 0, hi = su.ntb - 1;   // target block of unit u
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (su.off[mid] <= u) lo = mid; else hi = mid - 1;
    }
    const int tb = lo, fb = su.first_body(tb);
    const int seg_end = min(uend, su.off[tb + 1]);
    const int j0 = fb + (u - su.off[tb]), j1 = fb + (seg_end - su.off[tb]);
    const int slot = c - su.cta_of(su.off[tb]);
    u = seg_end;

    int pp[2], pb[2];
    float xp[2][3], wq[2][3];
    float4 cih[2], cil[2];
    float2 nf[2][3];
    float sacc[2][3], kacc[2][3];
#pragma unroll
    for (int t = 0; t < 2; t++) {
      const int p = tb * SYM_TB + t * SYM_THREADS + threadIdx.x;
      pp[t] = p;
      const int pc = p < N ? p : N - 1;
      const int bi = pc / ns, qi = pc - bi * ns;
      pb[t] = p < N ? bi : 0x7fffffff;
      for (int d = 0; d < 3; d++) {
        xp[t][d] = tmpl32[d * ns + qi];
        wq[t][d] = tmpl32[(3 + d) * ns + qi];
        const float f = phi32[3 * pc + d];
        nf[t][d] = make_float2(-f, -f);
        sacc[t][d] = 0.f;
        kacc[t][d] = 0.f;
      }
      cih[t] = *reinterpret_cast<const float4*>(c32 + 8 * bi);
      cil[t] = *reinterpret_cast<const float4*>(c32 + 8 * bi + 4);
    }
    for (int jc = j0; jc < j1; jc += SYM_CHUNK) {
      const int nb = min(SYM_CHUNK, j1 - jc);
      __syncthreads();
      const int cnt = nb * ns;
      const float* src = phi32 + 3 * (size_t)jc * ns;
      for (int t = threadIdx.x; t < 3 * cnt; t += blockDim.x) {
        const int node = t / 3, d = t - 3 * node;
        const int b = node / ns, q = node - b * ns;
        s_f[(d * SYM_CHUNK + b) * ns_pad + q] = src[t];
      }
      for (int t = threadIdx.x; t < nb * (ns_pad - ns); t += blockDim.x) {
        const int b = t / (ns_pad - ns), q = ns + t % (ns_pad - ns);
        for (int d = 0; d < 3; d++) s_f[(d * SYM_CHUNK + b) * ns_pad + q] = 0.f;
      }
      __syncthreads();
      for (int b = 0; b < nb; b++) {
        const int j = jc + b;
        const bool any_rev = j > fb;   // the same for the whole CTA
        const float4 cjh = *reinterpret_cast<const float4*>(c32 + 8 * j);
        const float4 cjl = *reinterpret_cast<const float4*>(c32 + 8 * j + 4);
        float2 e[2][3], wp[2][3], acc[2][3];
#pragma unroll
        for (int t = 0; t < 2; t++) {
          const float ex = ((cih[t].x - cjh.x) + (cil[t].x - cjl.x)) + xp[t][0];
          const float ey = ((cih[t].y - cjh.y) + (cil[t].y - cjl.y)) + xp[t][1];
          const float ez = ((cih[t].z - cjh.z) + (cil[t].z - cjl.z)) + xp[t][2];
          e[t][0] = make_float2(ex, ex);
          e[t][1] = make_float2(ey, ey);
          e[t][2] = make_float2(ez, ez);
          const float rm = pb[t] < j ? 1.f : 0.f;   // reverse only for bodies before j
          for (int d = 0; d < 3; d++) {
            wp[t][d] = make_float2(rm * wq[t][d], rm * wq[t][d]);
            acc[t][d] = make_float2(0.f, 0.f);
          }
        }
        const float* fxb = s_f + (0 * SYM_CHUNK + b) * ns_pad;
        const float* fyb = s_f + (1 * SYM_CHUNK + b) * ns_pad;
        const float* fzb = s_f + (2 * SYM_CHUNK + b) * ns_pad;
        float* rout = s_rev + (size_t)(buf * SYM_WARPS + warp) * 3 * ns_pad;
#pragma unroll 1
        for (int q = 0; q < ns_pad; q += 4) {
          const float4 X = *reinterpret_cast<const float4*>(s_nx + q);
          const float4 Y = *reinterpret_cast<const float4*>(s_ny + q);
          const float4 Z = *reinterpret_cast<const float4*>(s_nz + q);
          const float4 WX = *reinterpret_cast<const float4*>(s_wx + q);
          const float4 WY = *reinterpret_cast<const float4*>(s_wy + q);
          const float4 WZ = *reinterpret_cast<const float4*>(s_wz + q);
          const float4 FX = *reinterpret_cast<const float4*>(fxb + q);
          const float4 FY = *reinterpret_cast<const float4*>(fyb + q);
          const float4 FZ = *reinterpret_cast<const float4*>(fzb + q);
          float2 rv[2][3];
#pragma unroll
          for (int h = 0; h < 2; h++) {
            for (int d = 0; d < 3; d++) rv[h][d] = make_float2(0.f, 0.f);
            const float2 nx = h ? make_float2(X.z, X.w) : make_float2(X.x, X.y);
            const float2 ny = h ? make_float2(Y.z, Y.w) : make_float2(Y.x, Y.y);
            const float2 nz = h ? make_float2(Z.z, Z.w) : make_float2(Z.x, Z.y);
            const float2 wx = h ? make_float2(WX.z, WX.w) : make_float2(WX.x, WX.y);
            const float2 wy = h ? make_float2(WY.z, WY.w) : make_float2(WY.x, WY.y);
            const float2 wz = h ? make_float2(WZ.z, WZ.w) : make_float2(WZ.x, WZ.y);
            const float2 fx = h ? make_float2(FX.z, FX.w) : make_float2(FX.x, FX.y);
            const float2 fy = h ? make_float2(FY.z, FY.w) : make_float2(FY.x, FY.y);
            const float2 fz = h ? make_float2(FZ.z, FZ.w) : make_float2(FZ.x, FZ.y);
#pragma unroll
            for (int t = 0; t < 2; t++) sym_pair(e[t], nf[t], wp[t], nx, ny, nz, wx, wy, wz, fx, fy, fz, acc[t], rv[h]);
          }
          if (any_rev) {
            // value k = 6 h + 2 d + l is the reverse sum of source q + 2 h + l, component d
            float v[16];
#pragma unroll
            for (int h = 0; h < 2; h++)
              for (int d = 0; d < 3; d++) {
                v[6 * h + 2 * d] = rv[h][d].x;
                v[6 * h + 2 * d + 1] = rv[h][d].y;
              }
#pragma unroll
            for (int k = 12; k < 16; k++) v[k] = 0.f;
            const float tot = warp_transpose_sum16(v, lane);
            const int k = lane >> 1;
            if (!(lane & 1) && k < 12) {
              const int h = k / 6, d = (k - 6 * h) >> 1, l = k & 1;
              rout[d * ns_pad + q + 2 * h + l] = tot;
            }
          }
        }
#pragma unroll
        for (int t = 0; t < 2; t++)
          if (pb[t] <= j)
            for (int d = 0; d < 3; d++) kahan(sacc[t][d], kacc[t][d], acc[t][d].x + acc[t][d].y);
        if (any_rev) {
          __syncthreads();
          // sum the warps in order; row of unit (tb, j): [ns][3] floats
          float* dst = rev + su.roff[tb] + (size_t)(j - fb - 1) * 3 * ns;
          const float* sb = s_rev + (size_t)buf * SYM_WARPS * 3 * ns_pad;
          for (int k = threadIdx.x; k < 3 * ns; k += blockDim.x) {
            const int q = k / 3, d = k - 3 * q;
            float s = 0.f;
#pragma unroll
            for (int w = 0; w < SYM_WARPS; w++) s += sb[(w * 3 + d) * ns_pad + q];
            dst[k] = s;
          }
          buf ^= 1;
        }
      }
    }
#pragma unroll
    for (int t = 0; t < 2; t++)
      if (pp[t] < N) {
        double* o = partial + ((size_t)slot * N + pp[t]) * 3;
        for (int d = 0; d < 3; d++) o[d] = (double)sacc[t][d] - (double)kacc[t][d];
      }
  }
}

// out_p = forward partials + reverse rows of the target blocks before body(p)
// (in block order) + (P phi)_p.
__global__ void k_finish_sym(int N, int ns, int splits, const double* __restrict__ partial,
                             const float* __restrict__ rev, const long long* __restrict__ roff,
                             const double* __restrict__ coef, const double* __restrict__ tmpl64,
                             double* __restrict__ out) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= N) return;
  double a0 = 0.0, a1 = 0.0, a2 = 0.0;
  for (int s = 0; s < splits; s++) {
    const double* o = partial + ((size_t)s * N + p) * 3;
    a0 += o[0];
    a1 += o[1];
    a2 += o[2];
  }
  const int i = p / ns, q = p % ns;
  const int ntb_before = (int)(((long long)i * ns + SYM_TB - 1) / SYM_TB);   // blocks with first body < i
  for (int tb = 0; tb < ntb_before; tb++) {
    const int fb = (int)(((long long)tb * SYM_TB) / ns);
    const float* r = rev + roff[tb] + ((size_t)(i - fb - 1) * ns + q) * 3;
    a0 += (double)r[0];
    a1 += (double)r[1];
    a2 += (double)r[2];
  }
  const double* c = coef + 6 * i;
  const double* xi = tmpl64 + 8 * q;
  a0 += c[0] + (c[4] * xi[2] - c[5] * xi[1]);
  a1 += c[1] + (c[5] * xi[0] - c[3] * xi[2]);
  a2 += c[2] + (c[3] * xi[1] - c[4] * xi[0]);
  out[3 * p] = a0;
  out[3 * p + 1] = a1;
  out[3 * p + 2] = a2;
}

// ------------------------------------------------------------------ host side
static size_t sym_smem(int ns) {
  const int ns_pad = (ns + 3) & ~3;
  return sizeof(float) * ((size_t)6 * ns_pad + 3 * SYM_CHUNK * ns_pad + 2 * SYM_WARPS * 3 * ns_pad);
}

static int host_cta_of(long long u, int U, int G) {
  auto start = [&](long long c) { return (c * U) / G; };
  long long c = (u * G) / U;
  while (c + 1 < G && start(c + 1) <= u) c++;
  while (c > 0 && start(c) > u) c--;
  return (int)c;
}

// Unit offsets, reverse-row offsets, one-wave grid, partial slots and the
// reverse buffer (once per context; the body count and grid never change).
int stokes_sym_configure(lcp_ctx* ctx) {
  const int N = ctx->N, ns = ctx->ns, M = ctx->M;
  const size_t smem = sym_smem(ns);
  if (smem > 48 * 1024)
    LCP_CUDA(cudaFuncSetAttribute(k_pair32_sym, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  LCP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ctx->occsym, k_pair32_sym, SYM_THREADS, smem));
  const int ntb = (N + SYM_TB - 1) / SYM_TB;
  std::vector<int> off(ntb + 1);
  std::vector<long long> roff(ntb + 1);
  off[0] = 0;
  roff[0] = 0;
  for (int tb = 0; tb < ntb; tb++) {
    const int fb = (int)(((long long)tb * SYM_TB) / ns);
    off[tb + 1] = off[tb] + (M - fb);
    roff[tb + 1] = roff[tb] + (long long)(M - 1 - fb) * 3 * ns;
  }
  const int U = off[ntb];
  int G = ctx->num_sms * (ctx->occsym > 0 ? ctx->occsym : 1);
  if (G > U) G = U;
  int slots = 1;
  for (int tb = 0; tb < ntb; tb++) {
    const int s = host_cta_of(off[tb + 1] - 1, U, G) - host_cta_of(off[tb], U, G) + 1;
    if (s > slots) slots = s;
  }
  ctx->sym_ntb = ntb;
  ctx->sym_units = U;
  ctx->sym_grid = G;
  ctx->sym_slots = slots;
  ctx->sym_off = (int*)ctx_alloc(ctx, sizeof(int) * (ntb + 1));
  ctx->sym_roff = (long long*)ctx_alloc(ctx, sizeof(long long) * (ntb + 1));
  ctx->sym_rev = (float*)ctx_alloc(ctx, sizeof(float) * (size_t)(roff[ntb] > 0 ? roff[ntb] : 1));
  if (!ctx->sym_off || !ctx->sym_roff || !ctx->sym_rev) return LCP_ERR_OOM;
  LCP_CUDA(cudaMemcpyAsync(ctx->sym_off, off.data(), sizeof(int) * (ntb + 1), cudaMemcpyHostToDevice, ctx->stream));
  LCP_CUDA(cudaMemcpyAsync(ctx->sym_roff, roff.data(), sizeof(long long) * (ntb + 1), cudaMemcpyHostToDevice,
                           ctx->stream));
  LCP_CUDA(cudaStreamSynchronize(ctx->stream));
  return LCP_OK;
}

// Bytes of the reverse buffer for a size (footprint estimate).
size_t stokes_sym_bytes(int M, int ns) {
  const long long N = (long long)M * ns;
  const long long ntb = (N + SYM_TB - 1) / SYM_TB;
  long long total = 0;
  for (long long tb = 0; tb < ntb; tb++) total += (long long)(M - 1 - (tb * SYM_TB) / ns) * 3 * ns;
  return sizeof(float) * (size_t)(total > 0 ? total : 1) + (sizeof(int) + sizeof(long long)) * (size_t)(ntb + 1);
}

// (K + P) phi with the symmetric FP32 pair sum; phi32 already holds phi in FP32.
int stokes_sym_apply(lcp_ctx* ctx, double* out) {
  const int N = ctx->N, ns = ctx->ns;
  const int ns_pad = (ns + 3) & ~3;
  if (ctx->sym_slots > ctx->splits) {
    ctx->err = "internal: symmetric pair-sum slots exceed the partial buffer";
    return LCP_ERR_INVALID_ARG;
  }
  LCP_CUDA(cudaMemsetAsync(ctx->partial, 0, sizeof(double) * 3 * (size_t)N * ctx->sym_slots, ctx->stream));
  SymUnits su{ctx->sym_units, ctx->sym_grid, ctx->sym_ntb, ns, ctx->sym_off, ctx->sym_roff};
  cudaEvent_t e0 = prof_begin(ctx);
  ++ctx->nlaunch, k_pair32_sym<<<ctx->sym_grid, SYM_THREADS, sym_smem(ns), ctx->stream>>>(
                      N, ns, ns_pad, su, ctx->tmpl32, ctx->centers32, ctx->phi32, ctx->partial, ctx->sym_rev);
  prof_end(ctx, e0, 0);
  ++ctx->nlaunch, k_finish_sym<<<(N + 255) / 256, 256, 0, ctx->stream>>>(
                      N, ns, ctx->sym_slots, ctx->partial, ctx->sym_rev, ctx->sym_roff, ctx->coef, ctx->tmpl64, out);
  LCP_CUDA(cudaGetLastError());
  return LCP_OK;
}
