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
// Work: target blocks of SYM_TB consecutive nodes times source bodies j >=
// the block's first body; a unit (tb, j) adds the forward terms of targets
// with body(p) <= j and the reverse terms of targets with body(p) < j.  Units
// are dealt in equal contiguous ranges to one wave of CTAs, as for the plain
// kernel.  Each thread holds four targets, packed two by two in FP32x2
// registers, and takes the sources one at a time (duplicated (v, v) pairs in
// shared memory).  Its four reverse contributions to a source are folded in
// registers, then summed over the warp (a transposing shuffle reduction) and
// over the CTA's warps in order, and written to a per-unit row of `rev`
// (FP32) that the finish kernel adds in target-block order.  Forward sums are
// FP64 per thread (shared memory) and go to partial[slot][p].  Everything is
// deterministic.
#include <cstring>
#include <vector>

#include "common.cuh"
#include "sym_units.cuh"

namespace {

constexpr int SYM_CHUNK = 2;                       // source bodies staged per tile
constexpr float SYM_EPS = 1e-20f;   // r = 0 only for q = p: keeps |r|^-3 = 1e30 finite, the term 0
// With |r|^-2 from a reciprocal, |r|^-4 = eps^-2 must stay finite at r = 0:
// 1e-12 perturbs |r|^2 >= 1e-2 (node spacing) by at most 1e-10 relative.
constexpr float SYM_EPS_RC = 1e-12f;

__device__ __forceinline__ float rsqrt_fast(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}


__device__ __forceinline__ float rcp_fast(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Two targets (the lanes of e, nf, wp) against one source (duplicated in the
// lanes of n*, w*, f*).  acc += forward terms, rv += reverse terms.  RC: take
// |r|^-2 from a second special-function reciprocal instead of squaring |r|^-1,
// one FP32x2 multiply fewer per pair (the special-function unit has room).
template <bool RC>
__device__ __forceinline__ void sym_pair(const float2 (&e)[3], const float2 (&nf)[3], const float2 (&wp)[3],
                                         float2 nx, float2 ny, float2 nz, float2 wx, float2 wy, float2 wz,
                                         float2 fx, float2 fy, float2 fz, float2 (&acc)[3], float2 (&rv)[3]) {
  const float2 rx = __fadd2_rn(e[0], nx);
  const float2 ry = __fadd2_rn(e[1], ny);
  const float2 rz = __fadd2_rn(e[2], nz);
  constexpr float eps = RC ? SYM_EPS_RC : SYM_EPS;
  float2 r2 = __ffma2_rn(rx, rx, make_float2(eps, eps));
  r2 = __ffma2_rn(ry, ry, r2);
  r2 = __ffma2_rn(rz, rz, r2);
  const float2 ir = make_float2(rsqrt_fast(r2.x), rsqrt_fast(r2.y));
  const float2 dx = __fadd2_rn(fx, nf[0]);
  const float2 dy = __fadd2_rn(fy, nf[1]);
  const float2 dz = __fadd2_rn(fz, nf[2]);
  float2 rd = __fmul2_rn(rx, dx);
  rd = __ffma2_rn(ry, dy, rd);
  rd = __ffma2_rn(rz, dz, rd);
  float2 t;
  if (RC) {
    // at r = 0 (a node with itself) rd = 0 and |r|^-4 = SYM_EPS_RC^-2 stays
    // finite, so t = 0
    const float2 i2 = make_float2(rcp_fast(r2.x), rcp_fast(r2.y));
    t = __fmul2_rn(__fmul2_rn(rd, ir), __fmul2_rn(i2, i2));
  } else {
    const float2 i2 = __fmul2_rn(ir, ir);
    t = __fmul2_rn(__fmul2_rn(rd, i2), __fmul2_rn(i2, ir));
  }
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

// Add a to the compensated sum (hi, lo) (Knuth's TwoSum: the rounding error of
// hi + a is recovered exactly and collected in lo).
__device__ __forceinline__ void two_sum_acc(float2& s, float a) {
  const float h = __fadd_rn(s.x, a);
  const float bp = __fsub_rn(h, s.x);
  const float err = __fadd_rn(__fsub_rn(s.x, __fsub_rn(h, bp)), __fsub_rn(a, bp));
  s.x = h;
  s.y = __fadd_rn(s.y, err);
}

// Sum NV values (NV = 8 or 16) over the 32 lanes of a warp: at each of the
// first log2(NV) levels a lane keeps half of its values and sends the other
// half to its partner (NV - 1 shuffles in all), then plain butterflies
// finish.  Afterwards lane l holds the warp total of value l / (32 / NV).
template <int NV>
__device__ __forceinline__ float warp_transpose_sum(const float (&v)[NV], int lane) {
  constexpr int LOG2NV = NV == 32 ? 5 : (NV == 16 ? 4 : 3);
  float a[NV];
#pragma unroll
  for (int i = 0; i < NV; i++) a[i] = v[i];
#pragma unroll
  for (int L = 0; L < LOG2NV; L++) {
    const int n = NV >> (L + 1), o = 16 >> L;
    const bool hi = lane & o;
#pragma unroll
    for (int i = 0; i < n; i++) {
      const float send = hi ? a[i] : a[i + n];
      const float keep = hi ? a[i + n] : a[i];
      a[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
#pragma unroll
  for (int o = 16 >> LOG2NV; o >= 1; o >>= 1) a[0] += __shfl_xor_sync(0xffffffffu, a[0], o);
  return a[0];
}

}  // namespace

// Kernel variants (autotuner candidates):
//   AOS:   shared-memory layout of the sources: per-component arrays of (v, v)
//          pairs, or one record per node read with 128-bit loads;
//   BATCH: sources per warp reduction (2 or 4);
//   MINB:  CTAs per SM the registers are sized for (4: 128, 3: 168 registers);
//   PIPE:  reduce the previous batch after computing the current one, so
//          the shuffle latency overlaps the arithmetic;
//   TPT, THR: targets per thread and CTA size (TPT x THR = SYM_TB);
//   CT:    source template (duplicated (v, v) pairs, AOS order) read from the
//          launch's parameter block `tpar` (constant bank: every lane reads the
//          same source) instead of shared memory;
//   RC:    |r|^-2 by a special-function reciprocal (see sym_pair);
//   CF:    forward sums carried across source bodies as compensated FP32
//          (hi, lo) pairs instead of FP64 adds (FP64 runs at 1/64 rate).
template <bool AOS, int BATCH, int MINB, bool PIPE, int TPT, int THR, bool CT, bool RC, bool CF>
__device__ __forceinline__ void pair32_sym_body(int N, int ns, int ns_pad, SymUnits su,
                                                const float* __restrict__ tmpl32, const float* __restrict__ c32,
                                                const float* __restrict__ phi32, double* __restrict__ partial,
                                                float* __restrict__ rev, const float2* tpar) {
  static_assert(!CT || AOS, "the parameter-block template is in record order");
  static_assert(TPT * THR == SYM_TB && TPT % 2 == 0, "a thread's targets fill FP32x2 packs of the block");
  constexpr int NPK = TPT / 2;       // FP32x2 packs of targets per thread
  constexpr int WARPS = THR / 32;
  // values per batch (3 per source) padded to a power of two for the transposing reduction
  constexpr int NV = 3 * BATCH <= 8 ? 8 : (3 * BATCH <= 16 ? 16 : 32);
  static_assert(3 * BATCH <= 32, "at most 32 values per warp reduction");
  constexpr int LPV = 32 / NV;   // lanes holding each reduced value
  extern __shared__ float4 smem4[];
  // AOS: s_t [ns_pad][3] float4 = (nx,nx,ny,ny) (nz,nz,wx,wx) (wy,wy,wz,wz);
  //      s_f [SYM_CHUNK][ns_pad][2] float4 = (fx,fx,fy,fy) (fz,fz,0,0)
  // SoA: s_t [6][ns_pad] float2; s_f [3][SYM_CHUNK][ns_pad] float2
  float2* s_t = reinterpret_cast<float2*>(smem4);
  float2* s_f = s_t + (CT ? 0 : 6 * ns_pad);
  const int f_len = AOS ? 4 * SYM_CHUNK * ns_pad : 3 * SYM_CHUNK * ns_pad;   // float2 entries
  float* s_rev = reinterpret_cast<float*>(s_f + f_len);                      // [WARPS][3][ns_pad]
  double* s_fwd = reinterpret_cast<double*>(s_rev + WARPS * 3 * ns_pad);       // [TPT][3][THR]
  float2* s_fwc = reinterpret_cast<float2*>(s_fwd);                              // CF: (hi, lo) in the same slots
  for (int q = threadIdx.x; q < (CT ? 0 : ns_pad); q += blockDim.x) {
    const bool real = q < ns;
    for (int d = 0; d < 3; d++) {
      const float x = real ? -tmpl32[d * ns + q] : (d == 0 ? -1.0e3f : 0.f);
      const float w = real ? tmpl32[(3 + d) * ns + q] : 0.f;
      if (AOS) {
        s_t[6 * q + d] = make_float2(x, x);
        s_t[6 * q + 3 + d] = make_float2(w, w);
      } else {
        s_t[d * ns_pad + q] = make_float2(x, x);
        s_t[(3 + d) * ns_pad + q] = make_float2(w, w);
      }
    }
  }
  if (AOS)   // pad slots of the density records stay zero
    for (int t = threadIdx.x; t < SYM_CHUNK * ns_pad; t += blockDim.x) s_f[4 * t + 3] = make_float2(0.f, 0.f);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c = blockIdx.x;
  int u = su.start(c);
  const int uend = su.start(c + 1);
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

    int pb[TPT], pq[TPT];   // body (INT_MAX past the end) and template node of each target
#pragma unroll
    for (int t = 0; t < TPT; t++) {
      const int p = tb * SYM_TB + t * THR + threadIdx.x;
      const int pc = p < N ? p : N - 1;
      const int bi = pc / ns;
      pb[t] = p < N ? bi : 0x7fffffff;
      pq[t] = pc - bi * ns;
      for (int d = 0; d < 3; d++) {
        if (CF) s_fwc[(t * 3 + d) * THR + threadIdx.x] = make_float2(0.f, 0.f);
        else s_fwd[(t * 3 + d) * THR + threadIdx.x] = 0.0;
      }
    }
    for (int jc = j0; jc < j1; jc += SYM_CHUNK) {
      const int nb = min(SYM_CHUNK, j1 - jc);
      __syncthreads();
      const int cnt = nb * ns;
      const float* src = phi32 + 3 * (size_t)jc * ns;
      for (int t = threadIdx.x; t < 3 * cnt; t += blockDim.x) {
        const int node = t / 3, d = t - 3 * node;
        const int b = node / ns, q = node - b * ns;
        const float v = src[t];
        s_f[AOS ? 4 * (b * ns_pad + q) + d : (d * SYM_CHUNK + b) * ns_pad + q] = make_float2(v, v);
      }
      for (int t = threadIdx.x; t < nb * (ns_pad - ns); t += blockDim.x) {
        const int b = t / (ns_pad - ns), q = ns + t % (ns_pad - ns);
        for (int d = 0; d < 3; d++)
          s_f[AOS ? 4 * (b * ns_pad + q) + d : (d * SYM_CHUNK + b) * ns_pad + q] = make_float2(0.f, 0.f);
      }
      __syncthreads();
      for (int b = 0; b < nb; b++) {
        const int j = jc + b;
        const bool any_rev = j > fb;   // the same for the whole CTA
        const float4 cjh = *reinterpret_cast<const float4*>(c32 + 8 * j);
        const float4 cjl = *reinterpret_cast<const float4*>(c32 + 8 * j + 4);
        // per pack k: targets 2k (lane x) and 2k+1 (lane y)
        float2 e[NPK][3], nf[NPK][3], wp[NPK][3], acc[NPK][3];
#pragma unroll
        for (int t = 0; t < TPT; t++) {
          const int k = t >> 1;
          const int bi = pb[t] == 0x7fffffff ? (N - 1) / ns : pb[t];
          const float4 cih = *reinterpret_cast<const float4*>(c32 + 8 * bi);
          const float4 cil = *reinterpret_cast<const float4*>(c32 + 8 * bi + 4);
          const int pc = bi * ns + pq[t];
          const float rm = pb[t] < j ? 1.f : 0.f;   // reverse only for bodies before j
          const float ev[3] = {((cih.x - cjh.x) + (cil.x - cjl.x)) + tmpl32[pq[t]],
                               ((cih.y - cjh.y) + (cil.y - cjl.y)) + tmpl32[ns + pq[t]],
                               ((cih.z - cjh.z) + (cil.z - cjl.z)) + tmpl32[2 * ns + pq[t]]};
#pragma unroll
          for (int d = 0; d < 3; d++) {
            const float nv = -phi32[3 * pc + d];
            const float wv = rm * tmpl32[(3 + d) * ns + pq[t]];
            if (t & 1) {
              e[k][d].y = ev[d];
              nf[k][d].y = nv;
              wp[k][d].y = wv;
              acc[k][d].y = 0.f;
            } else {
              e[k][d].x = ev[d];
              nf[k][d].x = nv;
              wp[k][d].x = wv;
              acc[k][d].x = 0.f;
            }
          }
        }
        float* rout = s_rev + (size_t)warp * 3 * ns_pad;
        float vp[NV];   // previous batch (PIPE)
        int qp = -1;
#pragma unroll 1
        for (int q = 0; q < ns_pad; q += BATCH) {
          float v[NV];
#pragma unroll
          for (int h = 0; h < BATCH; h++) {
            const int qq = q + h;
            float2 rv[3] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
            float2 nx, ny, nz, wx, wy, wz, fx, fy, fz;
            if (AOS) {
              const float4* t4 = reinterpret_cast<const float4*>(CT ? tpar : s_t) + 3 * qq;
              const float4 A = t4[0], B = t4[1], C = t4[2];
              nx = make_float2(A.x, A.y); ny = make_float2(A.z, A.w);
              nz = make_float2(B.x, B.y); wx = make_float2(B.z, B.w);
              wy = make_float2(C.x, C.y); wz = make_float2(C.z, C.w);
              const float4* f4 = reinterpret_cast<const float4*>(s_f) + 2 * (b * ns_pad + qq);
              const float4 F = f4[0], G = f4[1];
              fx = make_float2(F.x, F.y); fy = make_float2(F.z, F.w); fz = make_float2(G.x, G.y);
            } else {
              nx = s_t[qq]; ny = s_t[ns_pad + qq]; nz = s_t[2 * ns_pad + qq];
              wx = s_t[3 * ns_pad + qq]; wy = s_t[4 * ns_pad + qq]; wz = s_t[5 * ns_pad + qq];
              fx = s_f[(0 * SYM_CHUNK + b) * ns_pad + qq];
              fy = s_f[(1 * SYM_CHUNK + b) * ns_pad + qq];
              fz = s_f[(2 * SYM_CHUNK + b) * ns_pad + qq];
            }
#pragma unroll
            for (int k = 0; k < NPK; k++) sym_pair<RC>(e[k], nf[k], wp[k], nx, ny, nz, wx, wy, wz, fx, fy, fz, acc[k], rv);
#pragma unroll
            for (int d = 0; d < 3; d++) v[3 * h + d] = rv[d].x + rv[d].y;   // the thread's TPT targets
          }
#pragma unroll
          for (int k = 3 * BATCH; k < NV; k++) v[k] = 0.f;
          if (any_rev) {
            // value k = 3 h + d: reverse sum of source q + h, component d
            if (PIPE) {
              if (qp >= 0) {
                const float tot = warp_transpose_sum<NV>(vp, lane);
                const int k = lane / LPV;
                if (lane % LPV == 0 && k < 3 * BATCH) rout[(k % 3) * ns_pad + qp + k / 3] = tot;
              }
#pragma unroll
              for (int k = 0; k < NV; k++) vp[k] = v[k];
              qp = q;
            } else {
              const float tot = warp_transpose_sum<NV>(v, lane);
              const int k = lane / LPV;
              if (lane % LPV == 0 && k < 3 * BATCH) rout[(k % 3) * ns_pad + q + k / 3] = tot;
            }
          }
        }
        if (PIPE && any_rev && qp >= 0) {
          const float tot = warp_transpose_sum<NV>(vp, lane);
          const int k = lane / LPV;
          if (lane % LPV == 0 && k < 3 * BATCH) rout[(k % 3) * ns_pad + qp + k / 3] = tot;
        }
#pragma unroll
        for (int t = 0; t < TPT; t++)
          if (pb[t] <= j)
            for (int d = 0; d < 3; d++) {
              const float a = (t & 1) ? acc[t >> 1][d].y : acc[t >> 1][d].x;
              if (CF) two_sum_acc(s_fwc[(t * 3 + d) * THR + threadIdx.x], a);
              else s_fwd[(t * 3 + d) * THR + threadIdx.x] += (double)a;
            }
        if (any_rev) {
          __syncthreads();
          // sum the warps in order; row of unit (tb, j): [ns][3] floats
          float* dst = rev + su.roff[tb] + (size_t)(j - fb - 1) * 3 * ns;
          for (int k = threadIdx.x; k < 3 * ns; k += blockDim.x) {
            const int q = k / 3, d = k - 3 * q;
            float s = 0.f;
#pragma unroll
            for (int w = 0; w < WARPS; w++) s += s_rev[(w * 3 + d) * ns_pad + q];
            dst[k] = s;
          }
          __syncthreads();
        }
      }
    }
#pragma unroll
    for (int t = 0; t < TPT; t++) {
      const int p = tb * SYM_TB + t * THR + threadIdx.x;
      if (p < N) {
        double* o = partial + ((size_t)slot * N + p) * 3;
        for (int d = 0; d < 3; d++) {
          if (CF) {
            const float2 h = s_fwc[(t * 3 + d) * THR + threadIdx.x];
            o[d] = (double)h.x + (double)h.y;
          } else {
            o[d] = s_fwd[(t * 3 + d) * THR + threadIdx.x];
          }
        }
      }
    }
  }
}

#define PAIR32_SYM_VARIANT(NAME, AOS, BATCH, MINB, PIPE, TPT, THR)                                             \
  __global__ void __launch_bounds__(THR, MINB)                                                                  \
      NAME(int N, int ns, int ns_pad, SymUnits su, const float* __restrict__ tmpl32, const float* __restrict__ c32, \
           const float* __restrict__ phi32, double* __restrict__ partial, float* __restrict__ rev) {               \
    pair32_sym_body<AOS, BATCH, MINB, PIPE, TPT, THR, false, false, false>(N, ns, ns_pad, su, tmpl32, c32, phi32,  \
                                                                           partial, rev, nullptr);                 \
  }
// variants that take the source template from their parameter block
#define PAIR32_SYM_VARIANT_P(NAME, BATCH, MINB, TPT, THR, RC, CF)                                               \
  __global__ void __launch_bounds__(THR, MINB)                                                                  \
      NAME(int N, int ns, int ns_pad, SymUnits su, const float* __restrict__ tmpl32, const float* __restrict__ c32, \
           const float* __restrict__ phi32, double* __restrict__ partial, float* __restrict__ rev,                 \
           const __grid_constant__ SymTmplParam tp) {                                                              \
    pair32_sym_body<true, BATCH, MINB, false, TPT, THR, true, RC, CF>(N, ns, ns_pad, su, tmpl32, c32, phi32,      \
                                                                      partial, rev,                               \
                                                                      reinterpret_cast<const float2*>(tp.v));     \
  }
// Measured at 216 spheres x 242 nodes (ms per launch): sym_a4 1.69, sym_a4m4
// 1.67, sym_a8m2 1.70, sym_a2 1.75, sym 1.86, pipelined variants 1.84-1.96;
// the plain kernel 1.97.  At 64 spheres x 162 nodes: sym_a4 0.100, sym_a8m2
// 0.103, sym_a4m4 0.114 (plain 0.100).
PAIR32_SYM_VARIANT(k_pair32_sym_a4, true, 4, 3, false, 4, 128)
PAIR32_SYM_VARIANT(k_pair32_sym_a4m4, true, 4, 4, false, 4, 128)
PAIR32_SYM_VARIANT(k_pair32_sym_a8m2, true, 8, 2, false, 4, 128)
PAIR32_SYM_VARIANT(k_pair32_sym_a2, true, 2, 4, false, 4, 128)
PAIR32_SYM_VARIANT(k_pair32_sym, false, 2, 4, false, 4, 128)
// eight targets per thread (four FP32x2 packs) in CTAs of 64 threads: twice
// the independent chains per warp and half the reduction work per pair
// (216 spheres: t8b4 1.63, t8b2 1.65 ms)
PAIR32_SYM_VARIANT(k_pair32_sym_t8b2, true, 2, 4, false, 8, 64)
PAIR32_SYM_VARIANT(k_pair32_sym_t8b4, true, 4, 3, false, 8, 64)
// Template in the parameter block, |r|^-2 by reciprocal, compensated forward
// sums; measured at 216 spheres (ms): eight targets per thread 1.60 with the
// template alone, 1.57 with the reciprocal, 1.54 with both and the compensated
// sums (sym_p8rc, the default); four targets per thread 1.61 (sym_p4rc); two
// sources per reduction 1.69.
PAIR32_SYM_VARIANT_P(k_pair32_sym_p8rc, 4, 3, 8, 64, true, true)
PAIR32_SYM_VARIANT_P(k_pair32_sym_p4rc, 4, 3, 4, 128, true, true)
// five sources per reduction: 15 of the 16 reduced values are used (12 of 16 with four)
PAIR32_SYM_VARIANT_P(k_pair32_sym_p8rc5, 5, 3, 8, 64, true, true)

typedef void (*Pair32SymKernel)(int, int, int, SymUnits, const float*, const float*, const float*, double*, float*);
typedef void (*Pair32SymKernelP)(int, int, int, SymUnits, const float*, const float*, const float*, double*, float*,
                                 SymTmplParam);
struct Pair32SymVariant {
  Pair32SymKernel kernel;     // template from shared memory, or
  Pair32SymKernelP kernel_p;  // template from the parameter block
  bool aos;
  int batch;     // sources per warp reduction: node padding is a multiple of max(4, batch)
  int threads;   // CTA size; targets per thread = SYM_TB / threads
  const char* name;
};
static const Pair32SymVariant kSymVariants[] = {
    {k_pair32_sym_a4, nullptr, true, 4, 128, "sym_a4"},
    {k_pair32_sym_a4m4, nullptr, true, 4, 128, "sym_a4m4"},
    {k_pair32_sym_a8m2, nullptr, true, 8, 128, "sym_a8m2"},
    {k_pair32_sym_a2, nullptr, true, 2, 128, "sym_a2"},
    {k_pair32_sym, nullptr, false, 2, 128, "sym"},
    {k_pair32_sym_t8b2, nullptr, true, 2, 64, "sym_t8b2"},
    {k_pair32_sym_t8b4, nullptr, true, 4, 64, "sym_t8b4"},
    {nullptr, k_pair32_sym_p8rc, true, 4, 64, "sym_p8rc"},
    {nullptr, k_pair32_sym_p4rc, true, 4, 128, "sym_p4rc"},
    {nullptr, k_pair32_sym_p8rc5, true, 5, 64, "sym_p8rc5"}};
constexpr int kNumSymVariants = sizeof(kSymVariants) / sizeof(kSymVariants[0]);

// out_p = forward partials + reverse rows of the target blocks before body(p)
// (in block order) + (P phi)_p.  One thread per node component; the reverse
// rows are read four blocks at a time (independent loads in flight).
// rbase[tb] = roff[tb] - (first body of tb + 1) * 3 ns, so that the row of
// (tb, body i) starts at rbase[tb] + i * 3 ns (no division per row).
__global__ void k_finish_sym(int N, int ns, int splits, const double* __restrict__ partial,
                             const float* __restrict__ rev, const long long* __restrict__ rbase,
                             const double* __restrict__ coef, const double* __restrict__ tmpl64,
                             double* __restrict__ out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 3 * N) return;
  const int p = t / 3, d = t - 3 * p;
  double a = 0.0;
  for (int s = 0; s < splits; s++) a += partial[(size_t)s * 3 * N + t];
  const int i = p / ns, q = p - i * ns;
  const int nbefore = (i * ns + SYM_TB - 1) / SYM_TB;   // blocks whose first body is before i
  const long long within = (long long)i * 3 * ns + 3LL * q + d;
  // the FP32 reverse rows are summed as a compensated FP32 pair (TwoSum) and
  // converted once: FP64 adds run at 1/64 rate and dominated this kernel
  float2 rs = make_float2(0.f, 0.f);
  float r4[4];
  int tb = 0;
  for (; tb + 4 <= nbefore; tb += 4) {
#pragma unroll
    for (int u = 0; u < 4; u++) r4[u] = rev[rbase[tb + u] + within];
#pragma unroll
    for (int u = 0; u < 4; u++) two_sum_acc(rs, r4[u]);
  }
  for (; tb < nbefore; tb++) two_sum_acc(rs, rev[rbase[tb] + within]);
  a += (double)rs.x + (double)rs.y;
  const double* c = coef + 6 * i;
  const double* xi = tmpl64 + 8 * q;
  if (d == 0) a += c[0] + (c[4] * xi[2] - c[5] * xi[1]);
  else if (d == 1) a += c[1] + (c[5] * xi[0] - c[3] * xi[2]);
  else a += c[2] + (c[3] * xi[1] - c[4] * xi[0]);
  out[t] = a;
}

// ------------------------------------------------------------------ host side
static int sym_ns_pad(int ns, int v) {
  const int a = kSymVariants[v].batch > 4 ? kSymVariants[v].batch : 4;
  return (ns + a - 1) / a * a;
}

static size_t sym_smem(int ns, int v) {
  const int ns_pad = sym_ns_pad(ns, v);
  const bool aos = kSymVariants[v].aos;
  const size_t t_len = kSymVariants[v].kernel_p ? 0 : (size_t)6 * ns_pad;   // template in the parameter block
  return sizeof(float2) * (t_len + (aos ? 4 : 3) * SYM_CHUNK * ns_pad) +
         sizeof(float) * (kSymVariants[v].threads / 32) * 3 * ns_pad + sizeof(double) * 3 * SYM_TB;
}

int stokes_sym_df_configure(lcp_ctx* ctx, const int* off, int ntb);

// The reverse rows grow as N x M (about 0.7 KB per pair of bodies at 242
// nodes each): above a quarter of the device's memory the symmetric sums are
// left out and the plain kernels, whose buffers grow as N, serve the size.
static size_t sym_rev_cap() {
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return total_b / 4;
}

static int host_cta_of(long long u, int U, int G) {
  auto start = [&](long long c) { return (c * U) / G; };
  long long c = (u * G) / U;
  while (c + 1 < G && start(c + 1) <= u) c++;
  while (c > 0 && start(c) > u) c--;
  return (int)c;
}

// Unit offsets, reverse-row offsets, the reverse buffer, and per kernel
// variant the one-wave grid and its partial slots (once per context; the
// body count and grid never change).
int stokes_sym_configure(lcp_ctx* ctx) {
  const int N = ctx->N, ns = ctx->ns, M = ctx->M;
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
  ctx->sym_ntb = ntb;
  ctx->sym_units = U;
  ctx->sym_slots = 1;
  if (2 * sizeof(float) * (size_t)roff[ntb] > sym_rev_cap()) {   // every symmetric variant stays unusable
    ctx->sym = false;
    return LCP_OK;
  }
  // the source template as a launch parameter block (duplicated pairs, record order)
  const bool tparam_ok = ns <= SYM_TPARAM_NODES;
  if (tparam_ok) {
    std::vector<float> t32((size_t)6 * ns);
    LCP_CUDA(cudaMemcpyAsync(t32.data(), ctx->tmpl32, sizeof(float) * 6 * ns, cudaMemcpyDeviceToHost, ctx->stream));
    LCP_CUDA(cudaStreamSynchronize(ctx->stream));
    ctx->sym_tparam.assign(sizeof(SymTmplParam) / sizeof(float4), make_float4(0.f, 0.f, 0.f, 0.f));
    float2* tp = reinterpret_cast<float2*>(ctx->sym_tparam.data());
    for (int q = 0; q < SYM_TPARAM_NODES; q++) {
      const bool real = q < ns;
      for (int d = 0; d < 3; d++) {
        const float x = real ? -t32[(size_t)d * ns + q] : (d == 0 ? -1.0e3f : 0.f);
        const float w = real ? t32[(size_t)(3 + d) * ns + q] : 0.f;
        tp[6 * q + d] = make_float2(x, x);
        tp[6 * q + 3 + d] = make_float2(w, w);
      }
    }
  }
  for (int v = 0; v < kNumSymVariants && v < 16; v++) {
    const Pair32SymVariant& kv = kSymVariants[v];
    if (kv.kernel_p && !tparam_ok) {   // parameter-block variants cover up to SYM_TPARAM_NODES nodes
      ctx->symv_occ[v] = 0;
      continue;
    }
    const size_t smem = sym_smem(ns, v);
    const void* fn = kv.kernel_p ? (const void*)kv.kernel_p : (const void*)kv.kernel;
    if (smem > 48 * 1024) LCP_CUDA(raise_smem_limit(fn, smem));
    int occ = 0;
    if (kv.kernel_p)
      LCP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kv.kernel_p, kv.threads, smem));
    else
      LCP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kv.kernel, kv.threads, smem));
    int G = ctx->num_sms * (occ > 0 ? occ : 1);
    if (G > U) G = U;
    int slots = 1;
    for (int tb = 0; tb < ntb; tb++) {
      const int s = host_cta_of(off[tb + 1] - 1, U, G) - host_cta_of(off[tb], U, G) + 1;
      if (s > slots) slots = s;
    }
    ctx->symv_occ[v] = occ;
    ctx->symv_grid[v] = G;
    ctx->symv_slots[v] = slots;
    if (slots > ctx->sym_slots) ctx->sym_slots = slots;
  }
  const int df_slots = stokes_sym_df_configure(ctx, off.data(), ntb);
  if (df_slots > ctx->sym_slots) ctx->sym_slots = df_slots;
  // default: the symmetric sum when every CTA gets several units (otherwise
  // the one-wave balance of the plain kernel's finer units wins), in its
  // fastest measured form where that fits the size
  ctx->sym = U >= 4 * ctx->symv_grid[0];
  ctx->sym_v = 0;
  int v8 = -1, v85 = -1;
  for (int v = 0; v < kNumSymVariants && v < 16; v++) {
    if (std::strcmp(kSymVariants[v].name, "sym_p8rc") == 0 && ctx->symv_occ[v] > 0) v8 = v;
    if (std::strcmp(kSymVariants[v].name, "sym_p8rc5") == 0 && ctx->symv_occ[v] > 0) v85 = v;
  }
  // five sources per reduction save reduction work unless the padding of the
  // nodes to a multiple of five costs a CTA per SM (216 spheres x 242 nodes:
  // 1.518 vs 1.536 ms; 512 nodes per sphere: 1.93 vs 1.52 ms)
  if (v8 >= 0) ctx->sym_v = v8;
  if (v85 >= 0 && (v8 < 0 || ctx->symv_occ[v85] >= ctx->symv_occ[v8])) ctx->sym_v = v85;
  ctx->sym_off = (int*)ctx_alloc(ctx, sizeof(int) * (ntb + 1));
  ctx->sym_roff = (long long*)ctx_alloc(ctx, sizeof(long long) * (ntb + 1));
  ctx->sym_rbase = (long long*)ctx_alloc(ctx, sizeof(long long) * (ntb + 1));
  // room for double-float (hi, lo) rows: the symmetric double-float kernel shares the buffer
  ctx->sym_rev = (float*)ctx_alloc(ctx, 2 * sizeof(float) * (size_t)(roff[ntb] > 0 ? roff[ntb] : 1));
  if (!ctx->sym_off || !ctx->sym_roff || !ctx->sym_rbase || !ctx->sym_rev) return LCP_ERR_OOM;
  std::vector<long long> rbase(ntb + 1, 0);
  for (int tb = 0; tb < ntb; tb++)
    rbase[tb] = roff[tb] - (long long)((((long long)tb * SYM_TB) / ns) + 1) * 3 * ns;
  LCP_CUDA(cudaMemcpyAsync(ctx->sym_off, off.data(), sizeof(int) * (ntb + 1), cudaMemcpyHostToDevice, ctx->stream));
  LCP_CUDA(cudaMemcpyAsync(ctx->sym_roff, roff.data(), sizeof(long long) * (ntb + 1), cudaMemcpyHostToDevice,
                           ctx->stream));
  LCP_CUDA(cudaMemcpyAsync(ctx->sym_rbase, rbase.data(), sizeof(long long) * (ntb + 1), cudaMemcpyHostToDevice,
                           ctx->stream));
  LCP_CUDA(cudaStreamSynchronize(ctx->stream));
  return LCP_OK;
}

int stokes_sym_variant_count() { return kNumSymVariants < 16 ? kNumSymVariants : 16; }
const char* stokes_sym_variant_name(int v) { return kSymVariants[v].name; }
bool stokes_sym_variant_usable(const lcp_ctx* ctx, int v) {
  return ctx->symv_occ[v] > 0 && ctx->symv_slots[v] <= ctx->splits;
}

// Bytes of the reverse buffer for a size (footprint estimate; 0 where the
// symmetric sums are left out).
size_t stokes_sym_bytes(int M, int ns) {
  const long long N = (long long)M * ns;
  const long long ntb = (N + SYM_TB - 1) / SYM_TB;
  long long total = 0;
  for (long long tb = 0; tb < ntb; tb++) total += (long long)(M - 1 - (tb * SYM_TB) / ns) * 3 * ns;
  if (2 * sizeof(float) * (size_t)total > sym_rev_cap()) return 0;
  return 2 * sizeof(float) * (size_t)(total > 0 ? total : 1) +
         (sizeof(int) + 2 * sizeof(long long)) * (size_t)(ntb + 1);
}

// (K + P) phi with the symmetric FP32 pair sum (variant ctx->sym_v); phi32
// already holds phi in FP32.
int stokes_sym_apply(lcp_ctx* ctx, double* out) {
  const int N = ctx->N, ns = ctx->ns;
  const int v = ctx->sym_v;
  const int ns_pad = sym_ns_pad(ns, v);
  if (!stokes_sym_variant_usable(ctx, v)) {
    ctx->err = "internal: symmetric pair-sum variant not usable for this size";
    return LCP_ERR_INVALID_ARG;
  }
  const int G = ctx->symv_grid[v], slots = ctx->symv_slots[v];
  LCP_CUDA(cudaMemsetAsync(ctx->partial, 0, sizeof(double) * 3 * (size_t)N * slots, ctx->stream));
  SymUnits su{ctx->sym_units, G, ctx->sym_ntb, ns, ctx->sym_off, ctx->sym_roff};
  cudaEvent_t e0 = prof_begin(ctx);
  const Pair32SymVariant& kv = kSymVariants[v];
  if (kv.kernel_p)
    ++ctx->nlaunch, kv.kernel_p<<<G, kv.threads, sym_smem(ns, v), ctx->stream>>>(
                        N, ns, ns_pad, su, ctx->tmpl32, ctx->centers32, ctx->phi32, ctx->partial, ctx->sym_rev,
                        *reinterpret_cast<const SymTmplParam*>(ctx->sym_tparam.data()));
  else
    ++ctx->nlaunch, kv.kernel<<<G, kv.threads, sym_smem(ns, v), ctx->stream>>>(
                        N, ns, ns_pad, su, ctx->tmpl32, ctx->centers32, ctx->phi32, ctx->partial, ctx->sym_rev);
  prof_end(ctx, e0, 0);
  ++ctx->nlaunch, k_finish_sym<<<(3 * N + 255) / 256, 256, 0, ctx->stream>>>(
                      N, ns, slots, ctx->partial, ctx->sym_rev, ctx->sym_rbase, ctx->coef, ctx->tmpl64, out);
  LCP_CUDA(cudaGetLastError());
  return LCP_OK;
}
