// Symmetric double-FP32 stresslet pair sum (the refinement residual of the
// mixed-precision mobility solve).
//
// The same pairing as the symmetric FP32 sum: for nodes on different bodies,
// with r = x_p - x_q and d = phi_q - phi_p, both ordered terms (Sec. 2, the
// double layer of the completed formulation) are (r . wn) t r with
// t = (r . d)/|r|^5 and wn the weighted normal of the source (forward) or of
// the target (reverse), so r, |r|^-5 and r . d in double-float arithmetic serve
// two terms.  Units, reverse rows and the finish step follow the FP32 kernel
// (sym_units.cuh); the reverse rows hold double-float (hi, lo) pairs.
//
// Each thread holds two targets in the lanes of FP32x2 double-float values
// (dfloat.cuh) and takes the sources one at a time from a shared-memory
// record of duplicated (v, v) pairs; the two reverse contributions are added
// in double-float, summed over the warp by a transposing shuffle reduction
// with double-float additions, and over the CTA's warps in order.
#include <vector>

#include "common.cuh"
#include "dfloat.cuh"
#include "sym_units.cuh"

namespace {

constexpr int SDF_THREADS = 256;   // two targets per thread: SYM_TB per CTA
constexpr int SDF_WARPS = SDF_THREADS / 32;
constexpr int SDF_CHUNK = 2;       // source bodies staged per tile
constexpr float SDF_EPS = 1e-20f;  // r = 0 only for q = p; the term is then 0
static_assert(2 * SDF_THREADS == SYM_TB, "two targets per thread");

__device__ __forceinline__ float rsqrt_mufu(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ D2 ddot3(const D2 (&a)[3], const D2 (&b)[3]) {
  return dadd_n(dadd_u(dmul_u(a[0], b[0]), dmul_u(a[1], b[1])), dmul_u(a[2], b[2]));
}

__device__ __forceinline__ D2 shfl_xor_d2(D2 v, int o) {
  D2 r;
  r.hi.x = __shfl_xor_sync(0xffffffffu, v.hi.x, o);
  r.hi.y = __shfl_xor_sync(0xffffffffu, v.hi.y, o);
  r.lo.x = __shfl_xor_sync(0xffffffffu, v.lo.x, o);
  r.lo.y = __shfl_xor_sync(0xffffffffu, v.lo.y, o);
  return r;
}

// Sum 8 double-float values over the warp; value k sits in pack k / 2, lane
// (x, y) = k % 2.  Transposing: the first two halving levels add whole packs
// (two independent double-float sums per FP32x2 instruction), the third splits
// the last pack, two butterflies finish; sums stay unnormalised until the end
// (lo grows by a few ulps of hi at most).  Lane l ends with value l / 4.
__device__ __forceinline__ dfl warp_transpose_sum8_packed(D2 (&P)[4], int lane) {
  {
    const bool up = lane & 16;   // keep values 4..7 (packs 2, 3), send 0..3
#pragma unroll
    for (int i = 0; i < 2; i++) {
      const D2 send = up ? P[i] : P[i + 2];
      const D2 keep = up ? P[i + 2] : P[i];
      P[i] = dadd_u(keep, shfl_xor_d2(send, 16));
    }
  }
  {
    const bool up = lane & 8;    // keep the second of the two remaining packs
    const D2 send = up ? P[0] : P[1];
    const D2 keep = up ? P[1] : P[0];
    P[0] = dadd_u(keep, shfl_xor_d2(send, 8));
  }
  const bool up = lane & 4;      // keep the odd value of the pack, send the even one
  const float sh = up ? P[0].hi.x : P[0].hi.y, sl = up ? P[0].lo.x : P[0].lo.y;
  const float kh = up ? P[0].hi.y : P[0].hi.x, kl = up ? P[0].lo.y : P[0].lo.x;
  D2 t = dadd_u({f2(kh), f2(kl)}, {f2(__shfl_xor_sync(0xffffffffu, sh, 4)), f2(__shfl_xor_sync(0xffffffffu, sl, 4))});
#pragma unroll
  for (int o = 2; o >= 1; o >>= 1)
    t = dadd_u(t, {f2(__shfl_xor_sync(0xffffffffu, t.hi.x, o)), f2(__shfl_xor_sync(0xffffffffu, t.lo.x, o))});
  t = fast2sum2(t.hi, t.lo);
  return {t.hi.x, t.lo.x};
}

}  // namespace

__global__ void __launch_bounds__(SDF_THREADS, 1)
k_pair_df_sym(int N, int ns, int ns_pad, SymUnits su, const double* __restrict__ tmpl64,
              const double* __restrict__ centers, const float* __restrict__ phidf, double* __restrict__ partial,
              float2* __restrict__ rev) {
  extern __shared__ float4 smem4[];
  // template record per node: (nx, nx, ny, ny | nz, nz, .. ) for -xi hi, -xi lo, wn hi, wn lo: 6 float4
  float4* s_t = smem4;
  // density record per (body, node): phi hi xyz, phi lo xyz duplicated: 3 float4
  float4* s_f = s_t + 6 * ns_pad;
  float2* s_rev = reinterpret_cast<float2*>(s_f + 3 * SDF_CHUNK * ns_pad);   // [warps][3][ns_pad] (hi, lo)
  double* s_fwd = reinterpret_cast<double*>(s_rev + SDF_WARPS * 3 * ns_pad);  // [2][3][threads]
  for (int q = threadIdx.x; q < ns_pad; q += blockDim.x) {
    const bool real = q < ns;
    float v[12];
    for (int d = 0; d < 3; d++) {
      const dfl x = real ? df_split(-tmpl64[8 * q + d]) : dfl{d == 0 ? -1.0e3f : 0.f, 0.f};
      const dfl w = real ? df_split(tmpl64[8 * q + 3 + d]) : dfl{0.f, 0.f};
      v[d] = x.hi;
      v[3 + d] = x.lo;
      v[6 + d] = w.hi;
      v[9 + d] = w.lo;
    }
    for (int k = 0; k < 6; k++) s_t[6 * q + k] = make_float4(v[2 * k], v[2 * k], v[2 * k + 1], v[2 * k + 1]);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c = blockIdx.x;
  int u = su.start(c);
  const int uend = su.start(c + 1);
  while (u < uend) {
    int lo = 0, hi = su.ntb - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (su.off[mid] <= u) lo = mid; else hi = mid - 1;
    }
    const int tb = lo, fb = su.first_body(tb);
    const int seg_end = min(uend, su.off[tb + 1]);
    const int j0 = fb + (u - su.off[tb]), j1 = fb + (seg_end - su.off[tb]);
    const int slot = c - su.cta_of(su.off[tb]);
    u = seg_end;

    int pb[2], pq[2];
#pragma unroll
    for (int t = 0; t < 2; t++) {
      const int p = tb * SYM_TB + t * SDF_THREADS + threadIdx.x;
      const int pc = p < N ? p : N - 1;
      const int bi = pc / ns;
      pb[t] = p < N ? bi : 0x7fffffff;
      pq[t] = pc - bi * ns;
      for (int d = 0; d < 3; d++) s_fwd[(t * 3 + d) * SDF_THREADS + threadIdx.x] = 0.0;
    }
    for (int jc = j0; jc < j1; jc += SDF_CHUNK) {
      const int nb = min(SDF_CHUNK, j1 - jc);
      __syncthreads();
      for (int t = threadIdx.x; t < nb * ns_pad; t += blockDim.x) {
        const int b = t / ns_pad, q = t - b * ns_pad;
        float v[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (q < ns) {
          const float* src = phidf + 6 * ((size_t)(jc + b) * ns + q);
          for (int k = 0; k < 6; k++) v[k] = src[k];
        }
        float4* rec = s_f + 3 * (b * ns_pad + q);
        rec[0] = make_float4(v[0], v[0], v[1], v[1]);
        rec[1] = make_float4(v[2], v[2], v[3], v[3]);
        rec[2] = make_float4(v[4], v[4], v[5], v[5]);
      }
      __syncthreads();
      for (int b = 0; b < nb; b++) {
        const int j = jc + b;
        const bool any_rev = j > fb;
        D2 E[3], NF[3], WP[3], ACC[3];
#pragma unroll
        for (int t = 0; t < 2; t++) {
          const int bi = pb[t] == 0x7fffffff ? (N - 1) / ns : pb[t];
          const int pc = bi * ns + pq[t];
          const float rm = pb[t] < j ? 1.f : 0.f;
#pragma unroll
          for (int d = 0; d < 3; d++) {
            const dfl e = df_split((centers[3 * bi + d] - centers[3 * j + d]) + tmpl64[8 * pq[t] + d]);
            const dfl w = df_split(tmpl64[8 * pq[t] + 3 + d]);
            const float fh = phidf[6 * (size_t)pc + d], fl = phidf[6 * (size_t)pc + 3 + d];
            if (t) {
              E[d].hi.y = e.hi; E[d].lo.y = e.lo;
              NF[d].hi.y = -fh; NF[d].lo.y = -fl;
              WP[d].hi.y = rm * w.hi; WP[d].lo.y = rm * w.lo;
              ACC[d].hi.y = 0.f; ACC[d].lo.y = 0.f;
            } else {
              E[d].hi.x = e.hi; E[d].lo.x = e.lo;
              NF[d].hi.x = -fh; NF[d].lo.x = -fl;
              WP[d].hi.x = rm * w.hi; WP[d].lo.x = rm * w.lo;
              ACC[d].hi.x = 0.f; ACC[d].lo.x = 0.f;
            }
          }
        }
        float2* rout = s_rev + (size_t)warp * 3 * ns_pad;
#pragma unroll 1
        for (int q = 0; q < ns_pad; q += 2) {
          D2 RV[2][3];   // reverse terms of the two sources; lanes: the thread's two targets
#pragma unroll
          for (int h = 0; h < 2; h++) {
            const int qq = q + h;
            const float4* tr = s_t + 6 * qq;
            const float4 A0 = tr[0], A1 = tr[1], A2 = tr[2], A3 = tr[3], A4 = tr[4], A5 = tr[5];
            // record order: xh x,y,z | xl x,y,z | wh x,y,z | wl x,y,z, two values per float4
            const D2 X[3] = {{make_float2(A0.x, A0.y), make_float2(A1.z, A1.w)},
                             {make_float2(A0.z, A0.w), make_float2(A2.x, A2.y)},
                             {make_float2(A1.x, A1.y), make_float2(A2.z, A2.w)}};
            const D2 W[3] = {{make_float2(A3.x, A3.y), make_float2(A4.z, A4.w)},
                             {make_float2(A3.z, A3.w), make_float2(A5.x, A5.y)},
                             {make_float2(A4.x, A4.y), make_float2(A5.z, A5.w)}};
            const float4* fr = s_f + 3 * (b * ns_pad + qq);
            const float4 B0 = fr[0], B1 = fr[1], B2 = fr[2];
            // record order: phi hi x,y,z | phi lo x,y,z
            const D2 F[3] = {{make_float2(B0.x, B0.y), make_float2(B1.z, B1.w)},
                             {make_float2(B0.z, B0.w), make_float2(B2.x, B2.y)},
                             {make_float2(B1.x, B1.y), make_float2(B2.z, B2.w)}};
            D2 R[3];
#pragma unroll
            for (int d = 0; d < 3; d++) R[d] = dadd_n(E[d], X[d]);
            D2 r2 = dadd_u(dadd_u(dsq_u(R[0]), dsq_u(R[1])), dsq_u(R[2]));
            r2.hi = add2(r2.hi, f2(SDF_EPS));
            const float2 y0 = make_float2(rsqrt_mufu(r2.hi.x), rsqrt_mufu(r2.hi.y));
            const float2 yy = mul2(y0, y0);
            const D2 tt = dmul_u(r2, {yy, fma2(y0, y0, neg2(yy))});
            const float2 hh = sub2(sub2(f2(1.f), tt.hi), tt.lo);
            const D2 ir = fast2sum2(y0, mul2(mul2(f2(0.5f), y0), hh));
            const D2 i2 = dsq_u(ir);
            D2 Dd[3];
#pragma unroll
            for (int d = 0; d < 3; d++) Dd[d] = dadd_u(F[d], NF[d]);
            const D2 rd = ddot3(R, Dd);
            const D2 tq = dmul_u(dmul_u(rd, i2), dmul_u(i2, ir));
            const D2 rq = ddot3(R, W);
            const D2 rp = ddot3(R, WP);
            const D2 sf = dmul_u(rq, tq);
            const D2 sr = dmul_u(rp, tq);
#pragma unroll
            for (int d = 0; d < 3; d++) {
              ACC[d] = dadd_n(ACC[d], dmul_u(sf, R[d]));
              RV[h][d] = dmul_u(sr, R[d]);
            }
          }
          if (any_rev) {
            // fold the thread's two targets, both sources at once: pack d = component d of
            // (source q, source q + 1), i.e. value k = 2 d + h
            D2 P[4];
#pragma unroll
            for (int d = 0; d < 3; d++)
              P[d] = dadd_u({make_float2(RV[0][d].hi.x, RV[1][d].hi.x), make_float2(RV[0][d].lo.x, RV[1][d].lo.x)},
                            {make_float2(RV[0][d].hi.y, RV[1][d].hi.y), make_float2(RV[0][d].lo.y, RV[1][d].lo.y)});
            P[3] = {f2(0.f), f2(0.f)};
            const dfl tot = warp_transpose_sum8_packed(P, lane);
            const int k = lane >> 2;
            if (!(lane & 3) && k < 6) rout[(k >> 1) * ns_pad + q + (k & 1)] = make_float2(tot.hi, tot.lo);
          }
        }
#pragma unroll
        for (int t = 0; t < 2; t++)
          if (pb[t] <= j)
            for (int d = 0; d < 3; d++) {
              const double a = t ? (double)ACC[d].hi.y + (double)ACC[d].lo.y : (double)ACC[d].hi.x + (double)ACC[d].lo.x;
              s_fwd[(t * 3 + d) * SDF_THREADS + threadIdx.x] += a;
            }
        if (any_rev) {
          __syncthreads();
          float2* dst = rev + su.roff[tb] + (size_t)(j - fb - 1) * 3 * ns;
          for (int k = threadIdx.x; k < 3 * ns; k += blockDim.x) {
            const int q = k / 3, d = k - 3 * q;
            dfl s{0.f, 0.f};
            for (int w = 0; w < SDF_WARPS; w++) {
              const float2 r = s_rev[(w * 3 + d) * ns_pad + q];
              s = df_add(s, dfl{r.x, r.y});
            }
            dst[k] = make_float2(s.hi, s.lo);
          }
          __syncthreads();
        }
      }
    }
#pragma unroll
    for (int t = 0; t < 2; t++) {
      const int p = tb * SYM_TB + t * SDF_THREADS + threadIdx.x;
      if (p < N) {
        double* o = partial + ((size_t)slot * N + p) * 3;
        for (int d = 0; d < 3; d++) o[d] = s_fwd[(t * 3 + d) * SDF_THREADS + threadIdx.x];
      }
    }
  }
}

// out_p = forward partials + the double-float reverse rows of the target
// blocks before body(p) (in block order) + (P phi)_p; one thread per component.
__global__ void k_finish_sym_df(int N, int ns, int splits, const double* __restrict__ partial,
                                const float2* __restrict__ rev, const long long* __restrict__ rbase,
                                const double* __restrict__ coef, const double* __restrict__ tmpl64,
                                double* __restrict__ out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 3 * N) return;
  const int p = t / 3, d = t - 3 * p;
  double a = 0.0;
  for (int s = 0; s < splits; s++) a += partial[(size_t)s * 3 * N + t];
  const int i = p / ns, q = p - i * ns;
  const int nbefore = (i * ns + SYM_TB - 1) / SYM_TB;
  const long long within = (long long)i * 3 * ns + 3LL * q + d;
  for (int tb = 0; tb < nbefore; tb++) {   // rows at rbase[tb] + i * 3 ns (see k_finish_sym)
    const float2 r = rev[rbase[tb] + within];
    a += (double)r.x + (double)r.y;
  }
  const double* c = coef + 6 * i;
  const double* xi = tmpl64 + 8 * q;
  if (d == 0) a += c[0] + (c[4] * xi[2] - c[5] * xi[1]);
  else if (d == 1) a += c[1] + (c[5] * xi[0] - c[3] * xi[2]);
  else a += c[2] + (c[3] * xi[1] - c[4] * xi[0]);
  out[t] = a;
}

// ------------------------------------------------------------------ host side
static int sdf_ns_pad(int ns) { return (ns + 1) & ~1; }

static size_t sdf_smem(int ns) {
  const int ns_pad = sdf_ns_pad(ns);
  return sizeof(float4) * ((size_t)6 * ns_pad + 3 * SDF_CHUNK * ns_pad) + sizeof(float2) * SDF_WARPS * 3 * ns_pad +
         sizeof(double) * 2 * 3 * SDF_THREADS;
}

static int host_cta_of_df(long long u, int U, int G) {
  auto start = [&](long long c) { return (c * U) / G; };
  long long c = (u * G) / U;
  while (c + 1 < G && start(c + 1) <= u) c++;
  while (c > 0 && start(c) > u) c--;
  return (int)c;
}

// Grid and partial slots of the double-float kernel on the symmetric units
// (off: [ntb + 1] host copy).  Returns the slots it needs (0 if it cannot run).
int stokes_sym_df_configure(lcp_ctx* ctx, const int* off, int ntb) {
  const size_t smem = sdf_smem(ctx->ns);
  if (smem > 227 * 1024) return 0;
  if (smem > 48 * 1024) LCP_CUDA(raise_smem_limit((const void*)k_pair_df_sym, smem));
  int occ = 0;
  LCP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_pair_df_sym, SDF_THREADS, smem));
  if (occ <= 0) return 0;
  const int U = off[ntb];
  int G = ctx->num_sms * occ;
  if (G > U) G = U;
  int slots = 1;
  for (int tb = 0; tb < ntb; tb++) {
    const int s = host_cta_of_df(off[tb + 1] - 1, U, G) - host_cta_of_df(off[tb], U, G) + 1;
    if (s > slots) slots = s;
  }
  ctx->symdf_grid = G;
  ctx->symdf_slots = slots;
  return slots;
}

// (K + P) phi with the symmetric double-float pair sum; phidf already holds
// phi split into hi/lo floats.
int stokes_sym_df_apply(lcp_ctx* ctx, double* out) {
  const int N = ctx->N, ns = ctx->ns;
  const int G = ctx->symdf_grid, slots = ctx->symdf_slots;
  if (G <= 0 || slots > ctx->splits) {
    ctx->err = "internal: symmetric double-float pair sum not configured";
    return LCP_ERR_INVALID_ARG;
  }
  LCP_CUDA(cudaMemsetAsync(ctx->partial, 0, sizeof(double) * 3 * (size_t)N * slots, ctx->stream));
  SymUnits su{ctx->sym_units, G, ctx->sym_ntb, ns, ctx->sym_off, ctx->sym_roff};
  float2* rev = reinterpret_cast<float2*>(ctx->sym_rev);
  cudaEvent_t e0 = prof_begin(ctx);
  ++ctx->nlaunch, k_pair_df_sym<<<G, SDF_THREADS, sdf_smem(ns), ctx->stream>>>(
                      N, ns, sdf_ns_pad(ns), su, ctx->tmpl64, ctx->centers, ctx->phidf, ctx->partial, rev);
  prof_end(ctx, e0, 2);
  ++ctx->nlaunch, k_finish_sym_df<<<(3 * N + 255) / 256, 256, 0, ctx->stream>>>(
                      N, ns, slots, ctx->partial, rev, ctx->sym_rbase, ctx->coef, ctx->tmpl64, out);
  LCP_CUDA(cudaGetLastError());
  return LCP_OK;
}
