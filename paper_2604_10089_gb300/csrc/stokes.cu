// Boundary-integral operator kernels: the stresslet pair sum K (the hot path),
// the rigid projector P, the Stokeslet/rotlet right-hand side and the rigid
// velocities.  Sec. 2 / Fig. 1 of the paper: M ~ P M_stk P^T, where every
// application of M_stk is a GMRES solve whose iterations apply K + P.
//
//   (K phi)_p = sum_{q != p} w_q T(x_p - x_q, n_q)(phi_q - phi_p),
//   T(r, n) v = -(3 / 4 pi) r (r . n)(r . v) / |r|^5.
//
// Layout: node vectors [N][3] FP64, body-major.  All spheres share one
// quadrature template, so a source tile is one body: the template (xi, w n)
// stays in shared memory for the whole kernel and only the density of the
// source body is staged per tile.  Positions are body-relative,
// r = ((c_i - c_j) + xi_p) - xi_q with c_i - c_j formed from hi/lo parts,
// which keeps FP32 differences accurate for nodes of touching spheres.
#include <cmath>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "dfloat.cuh"

namespace {

constexpr int PAIR_THREADS = PAIR_THREADS_PUBLIC;
constexpr int PAIR_CHUNK = PAIR_CHUNK_PUBLIC;   // source bodies staged per shared-memory tile
constexpr float EPS32 = 1e-30f;   // r = 0 only for q = p; then rn = rd = 0 and the term is 0
constexpr double EPS64 = 1e-300;

__device__ __forceinline__ float rsqrt_approx(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ void kahan_add(float& s, float& c, float v) {
  const float y = v - c;
  const float t = s + y;
  c = (t - s) - y;
  s = t;
}

}  // namespace

// FP32 stresslet sum: two targets per thread (PAIR32_TARGETS per CTA), sources
// two at a time in packed FP32x2 arithmetic, |r|^-2 as the square of the MUFU
// reciprocal square root.  Per-body (tile) sums in FP32, Kahan-compensated
// FP32 across tiles, written as FP64 partials partial[slot][p][3].  ns_pad is
// ns rounded up to 4; padded sources carry zero weight.
__device__ __forceinline__ void pair2(const float2 ex, const float2 ey, const float2 ez,
                                      const float2 nfx, const float2 nfy, const float2 nfz,
                                      const float4& X, const float4& Y, const float4& Z,
                                      const float4& WX, const float4& WY, const float4& WZ,
                                      const float4& FX, const float4& FY, const float4& FZ, bool upper,
                                      float2& ax, float2& ay, float2& az) {
  const float2 eps = make_float2(EPS32, EPS32);
  const float2 nxq = upper ? make_float2(X.z, X.w) : make_float2(X.x, X.y);
  const float2 nyq = upper ? make_float2(Y.z, Y.w) : make_float2(Y.x, Y.y);
  const float2 nzq = upper ? make_float2(Z.z, Z.w) : make_float2(Z.x, Z.y);
  const float2 wx = upper ? make_float2(WX.z, WX.w) : make_float2(WX.x, WX.y);
  const float2 wy = upper ? make_float2(WY.z, WY.w) : make_float2(WY.x, WY.y);
  const float2 wz = upper ? make_float2(WZ.z, WZ.w) : make_float2(WZ.x, WZ.y);
  const float2 fx = upper ? make_float2(FX.z, FX.w) : make_float2(FX.x, FX.y);
  const float2 fy = upper ? make_float2(FY.z, FY.w) : make_float2(FY.x, FY.y);
  const float2 fz = upper ? make_float2(FZ.z, FZ.w) : make_float2(FZ.x, FZ.y);
  const float2 rx = __fadd2_rn(ex, nxq);
  const float2 ry = __fadd2_rn(ey, nyq);
  const float2 rz = __fadd2_rn(ez, nzq);
  float2 r2 = __ffma2_rn(rx, rx, eps);
  r2 = __ffma2_rn(ry, ry, r2);
  r2 = __ffma2_rn(rz, rz, r2);
  const float2 ir = make_float2(rsqrt_approx(r2.x), rsqrt_approx(r2.y));
  const float2 i2 = __fmul2_rn(ir, ir);
  float2 rn = __fmul2_rn(rx, wx);
  rn = __ffma2_rn(ry, wy, rn);
  rn = __ffma2_rn(rz, wz, rn);
  const float2 dx = __fadd2_rn(fx, nfx);
  const float2 dy = __fadd2_rn(fy, nfy);
  const float2 dz = __fadd2_rn(fz, nfz);
  float2 rd = __fmul2_rn(rx, dx);
  rd = __ffma2_rn(ry, dy, rd);
  rd = __ffma2_rn(rz, dz, rd);
  const float2 s = __fmul2_rn(__fmul2_rn(__fmul2_rn(rn, i2), __fmul2_rn(rd, i2)), ir);
  ax = __ffma2_rn(s, rx, ax);
  ay = __ffma2_rn(s, ry, ay);
  az = __ffma2_rn(s, rz, az);
}

template <int TPT, int CH>
__device__ __forceinline__ void pair32_body(int N, int ns, int ns_pad, Units un, const float* __restrict__ tmpl32,
                                            const float* __restrict__ c32, const float* __restrict__ phi32,
                                            double* __restrict__ partial) {
  extern __shared__ float4 smem4[];
  float* sm = reinterpret_cast<float*>(smem4);
  float* s_nx = sm;                    // -xi, per template node (padded)
  float* s_ny = s_nx + ns_pad;
  float* s_nz = s_ny + ns_pad;
  float* s_wx = s_nz + ns_pad;         // -(3/4pi) w n
  float* s_wy = s_wx + ns_pad;
  float* s_wz = s_wy + ns_pad;
  float* s_f = s_wz + ns_pad;          // [3][CH][ns_pad] source densities

  for (int q = threadIdx.x; q < ns_pad; q += blockDim.x) {
    const bool real = q < ns;
    s_nx[q] = real ? -tmpl32[q] : -1.0e3f;
    s_ny[q] = real ? -tmpl32[ns + q] : 0.f;
    s_nz[q] = real ? -tmpl32[2 * ns + q] : 0.f;
    s_wx[q] = real ? tmpl32[3 * ns + q] : 0.f;
    s_wy[q] = real ? tmpl32[4 * ns + q] : 0.f;
    s_wz[q] = real ? tmpl32[5 * ns + q] : 0.f;
  }
  const int M = un.M;
  const int c = blockIdx.x;
  int u = un.start(c);
  const int uend = un.start(c + 1);
  while (u < uend) {
    const int tb = u / M, jb0 = u - tb * M;
    const int jb1 = min(M, jb0 + (uend - u));
    const int slot = c - un.first_cta(tb);
    u += jb1 - jb0;
    int pp[TPT];
    float xp[TPT][3];
    float4 cih[TPT], cil[TPT];
    float2 nf[TPT][3];
    float sacc[TPT][3], kacc[TPT][3];
#pragma unroll
    for (int t = 0; t < TPT; t++) {
      const int p = tb * (TPT * PAIR_THREADS) + t * PAIR_THREADS + threadIdx.x;
      pp[t] = p;
      const int pc = p < N ? p : N - 1;
      const int bi = pc / ns, qi = pc - bi * ns;
      xp[t][0] = tmpl32[qi];
      xp[t][1] = tmpl32[ns + qi];
      xp[t][2] = tmpl32[2 * ns + qi];
      cih[t] = *reinterpret_cast<const float4*>(c32 + 8 * bi);
      cil[t] = *reinterpret_cast<const float4*>(c32 + 8 * bi + 4);
      for (int d = 0; d < 3; d++) {
        const float f = phi32[3 * pc + d];
        nf[t][d] = make_float2(-f, -f);
        sacc[t][d] = 0.f;
        kacc[t][d] = 0.f;
      }
    }
    for (int jc = jb0; jc < jb1; jc += CH) {
      const int nb = min(CH, jb1 - jc);
      __syncthreads();
      // stage densities of bodies jc .. jc+nb-1 (contiguous in phi32), SoA in smem
      const int cnt = nb * ns;
      const float* src = phi32 + 3 * (size_t)jc * ns;
      for (int t = threadIdx.x; t < 3 * cnt; t += blockDim.x) {
        const int node = t / 3, d = t - 3 * node;
        const int b = node / ns, q = node - b * ns;
        s_f[(d * CH + b) * ns_pad + q] = src[t];
      }
      for (int t = threadIdx.x; t < nb * (ns_pad - ns); t += blockDim.x) {
        const int b = t / (ns_pad - ns), q = ns + t % (ns_pad - ns);
        for (int d = 0; d < 3; d++) s_f[(d * CH + b) * ns_pad + q] = 0.f;
      }
      __syncthreads();
      for (int b = 0; b < nb; b++) {
        const int j = jc + b;
        const float4 cjh = *reinterpret_cast<const float4*>(c32 + 8 * j);
        const float4 cjl = *reinterpret_cast<const float4*>(c32 + 8 * j + 4);
        float2 e[TPT][3];
#pragma unroll
        for (int t = 0; t < TPT; t++) {
          const float ex = ((cih[t].x - cjh.x) + (cil[t].x - cjl.x)) + xp[t][0];
          const float ey = ((cih[t].y - cjh.y) + (cil[t].y - cjl.y)) + xp[t][1];
          const float ez = ((cih[t].z - cjh.z) + (cil[t].z - cjl.z)) + xp[t][2];
          e[t][0] = make_float2(ex, ex);
          e[t][1] = make_float2(ey, ey);
          e[t][2] = make_float2(ez, ez);
        }
        const float* fxb = s_f + (0 * CH + b) * ns_pad;
        const float* fyb = s_f + (1 * CH + b) * ns_pad;
        const float* fzb = s_f + (2 * CH + b) * ns_pad;
        float2 acc[TPT][3];
#pragma unroll
        for (int t = 0; t < TPT; t++)
          for (int d = 0; d < 3; d++) acc[t][d] = make_float2(0.f, 0.f);
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
#pragma unroll
          for (int t = 0; t < TPT; t++) {
            pair2(e[t][0], e[t][1], e[t][2], nf[t][0], nf[t][1], nf[t][2], X, Y, Z, WX, WY, WZ, FX, FY, FZ, false,
                  acc[t][0], acc[t][1], acc[t][2]);
            pair2(e[t][0], e[t][1], e[t][2], nf[t][0], nf[t][1], nf[t][2], X, Y, Z, WX, WY, WZ, FX, FY, FZ, true,
                  acc[t][0], acc[t][1], acc[t][2]);
          }
        }
#pragma unroll
        for (int t = 0; t < TPT; t++)
          for (int d = 0; d < 3; d++) kahan_add(sacc[t][d], kacc[t][d], acc[t][d].x + acc[t][d].y);
      }
    }
#pragma unroll
    for (int t = 0; t < TPT; t++)
      if (pp[t] < N) {
        double* o = partial + ((size_t)slot * N + pp[t]) * 3;
        for (int d = 0; d < 3; d++) o[d] = (double)sacc[t][d] - (double)kacc[t][d];
      }
  }
}

// The default FP32 kernel (two targets per thread, 8 source bodies per tile)
// and the variants the autotuner chooses from per size class.
__global__ void __launch_bounds__(PAIR_THREADS, 2)
k_pair32(int N, int ns, int ns_pad, Units un, const float* __restrict__ tmpl32, const float* __restrict__ c32,
         const float* __restrict__ phi32, double* __restrict__ partial) {
  pair32_body<PAIR32_TARGETS / PAIR_THREADS, PAIR_CHUNK>(N, ns, ns_pad, un, tmpl32, c32, phi32, partial);
}
#define PAIR32_VARIANT(NAME, TPT, CH, MINB)                                                                  \
  __global__ void __launch_bounds__(PAIR_THREADS, MINB)                                                       \
      NAME(int N, int ns, int ns_pad, Units un, const float* __restrict__ tmpl32, const float* __restrict__ c32, \
           const float* __restrict__ phi32, double* __restrict__ partial) {                                     \
    pair32_body<TPT, CH>(N, ns, ns_pad, un, tmpl32, c32, phi32, partial);                                       \
  }
PAIR32_VARIANT(k_pair32_t1c8, 1, 8, 4)
PAIR32_VARIANT(k_pair32_t2c16, 2, 16, 2)
PAIR32_VARIANT(k_pair32_t2c4, 2, 4, 2)
PAIR32_VARIANT(k_pair32_t1c16, 1, 16, 4)

typedef void (*Pair32Kernel)(int, int, int, Units, const float*, const float*, const float*, double*);
struct Pair32Variant {
  Pair32Kernel kernel;
  int tpt, chunk;
  const char* name;
};
static const Pair32Variant kPair32Variants[] = {
    {k_pair32, 2, 8, "t2c8"}, {k_pair32_t1c8, 1, 8, "t1c8"}, {k_pair32_t2c16, 2, 16, "t2c16"},
    {k_pair32_t2c4, 2, 4, "t2c4"}, {k_pair32_t1c16, 1, 16, "t1c16"}};
constexpr int kNumPair32Variants = sizeof(kPair32Variants) / sizeof(kPair32Variants[0]);

// ---------------------------------------------------------------------------
// Double-FP32 ("double-float") stresslet sum for the refinement residual; the
// arithmetic (TwoSum, TwoProd, Fast2Sum on hi + lo float pairs) is in dfloat.cuh.
__global__ void k_split_df(int L, const double* __restrict__ x, float* __restrict__ y) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= L) return;
  const int node = t / 3, d = t - 3 * node;
  const dfl v = df_split(x[t]);
  y[6 * node + d] = v.hi;
  y[6 * node + 3 + d] = v.lo;
}

// Double-float stresslet sum: same (target block, source body) decomposition
// as the FP32 kernel, one target per thread, source nodes two at a time in
// packed double-float arithmetic.  Shared memory holds the template as 12
// SoA arrays (-xi hi/lo, w n hi/lo per component) and the staged source
// densities as 6 SoA arrays per body (hi xyz, lo xyz).  ns_pad is ns rounded
// up to 4; padded sources have zero weight and density, far away.
__global__ void __launch_bounds__(PAIR_THREADS, 2)
k_pair_df(int N, int ns, int ns_pad, Units un, const double* __restrict__ tmpl64,
          const double* __restrict__ centers, const float* __restrict__ phidf, double* __restrict__ partial) {
  extern __shared__ float4 smem4[];
  float* sm = reinterpret_cast<float*>(smem4);
  float* s_t = sm;                       // [12][ns_pad]: -xi hi x,y,z; -xi lo x,y,z; wn hi x,y,z; wn lo x,y,z
  float* s_f = s_t + 12 * ns_pad;        // [6][PAIR_CHUNK][ns_pad]: phi hi x,y,z; phi lo x,y,z
  for (int q = threadIdx.x; q < ns_pad; q += blockDim.x) {
    const bool real = q < ns;
    for (int d = 0; d < 3; d++) {
      const dfl x = real ? df_split(-tmpl64[8 * q + d]) : dfl{d == 0 ? -1.0e3f : 0.f, 0.f};
      const dfl w = real ? df_split(tmpl64[8 * q + 3 + d]) : dfl{0.f, 0.f};
      s_t[d * ns_pad + q] = x.hi;
      s_t[(3 + d) * ns_pad + q] = x.lo;
      s_t[(6 + d) * ns_pad + q] = w.hi;
      s_t[(9 + d) * ns_pad + q] = w.lo;
    }
  }
  // padded source slots of every staged body stay zero for the whole kernel
  for (int t = threadIdx.x; t < 6 * PAIR_CHUNK * ns_pad; t += blockDim.x) s_f[t] = 0.f;
  const int M = un.M;
  const int c = blockIdx.x;
  const int fs = PAIR_CHUNK * ns_pad;
  int u = un.start(c);
  const int uend = un.start(c + 1);
  while (u < uend) {
    const int tb = u / M, jb0 = u - tb * M;
    const int jb1 = min(M, jb0 + (uend - u));
    const int slot = c - un.first_cta(tb);
    u += jb1 - jb0;
    const int p = tb * blockDim.x + threadIdx.x;
    const int pc = p < N ? p : N - 1;
    const int bi = pc / ns, qi = pc - bi * ns;
    const double xpx = tmpl64[8 * qi], xpy = tmpl64[8 * qi + 1], xpz = tmpl64[8 * qi + 2];
    const double cix = centers[3 * bi], ciy = centers[3 * bi + 1], ciz = centers[3 * bi + 2];
    const float* fp = phidf + 6 * (size_t)pc;
    const D2 nfx = {f2(-fp[0]), f2(-fp[3])}, nfy = {f2(-fp[1]), f2(-fp[4])}, nfz = {f2(-fp[2]), f2(-fp[5])};
    D2 ax = {f2(0.f), f2(0.f)}, ay = ax, az = ax;
    for (int jc = jb0; jc < jb1; jc += PAIR_CHUNK) {
      const int nb = min(PAIR_CHUNK, jb1 - jc);
      __syncthreads();
      const float* src = phidf + 6 * (size_t)jc * ns;
      for (int t = threadIdx.x; t < 6 * nb * ns; t += blockDim.x) {
        const int node = t / 6, k = t - 6 * node;         // k: 0..2 hi xyz, 3..5 lo xyz
        const int b = node / ns, q = node - b * ns;
        s_f[(k * PAIR_CHUNK + b) * ns_pad + q] = src[t];
      }
      __syncthreads();
      for (int b = 0; b < nb; b++) {
        const int j = jc + b;
        const dfl ex1 = df_split((cix - centers[3 * j]) + xpx);
        const dfl ey1 = df_split((ciy - centers[3 * j + 1]) + xpy);
        const dfl ez1 = df_split((ciz - centers[3 * j + 2]) + xpz);
        const D2 ex = {f2(ex1.hi), f2(ex1.lo)}, ey = {f2(ey1.hi), f2(ey1.lo)}, ez = {f2(ez1.hi), f2(ez1.lo)};
        const float* f = s_f + b * ns_pad;
#pragma unroll 1
        for (int q = 0; q < ns_pad; q += 2) {
#define LD2(ptr) (*reinterpret_cast<const float2*>((ptr) + q))
          const D2 rx = dadd_n(ex, {LD2(s_t), LD2(s_t + 3 * ns_pad)});
          const D2 ry = dadd_n(ey, {LD2(s_t + ns_pad), LD2(s_t + 4 * ns_pad)});
          const D2 rz = dadd_n(ez, {LD2(s_t + 2 * ns_pad), LD2(s_t + 5 * ns_pad)});
          D2 r2 = dadd_u(dadd_u(dsq_u(rx), dsq_u(ry)), dsq_u(rz));
          r2.hi = add2(r2.hi, f2(EPS32));
          // |r|^-1: MUFU seed y0, one Newton step y0 + (y0 / 2)(1 - r2 y0^2) in double-float
          const float2 y0 = make_float2(rsqrt_approx(r2.hi.x), rsqrt_approx(r2.hi.y));
          const float2 yy = mul2(y0, y0);
          const D2 t = dmul_u(r2, {yy, fma2(y0, y0, neg2(yy))});
          const float2 h = sub2(sub2(f2(1.f), t.hi), t.lo);
          // renormalised: an unnormalised lo of ~2^-22 y0 would drop lo^2 ~ 2^-44 in |r|^-2
          const D2 ir = fast2sum2(y0, mul2(mul2(f2(0.5f), y0), h));
          const D2 i2 = dsq_u(ir);
          const D2 rn = dadd_n(dadd_u(dmul_u(rx, {LD2(s_t + 6 * ns_pad), LD2(s_t + 9 * ns_pad)}),
                                      dmul_u(ry, {LD2(s_t + 7 * ns_pad), LD2(s_t + 10 * ns_pad)})),
                               dmul_u(rz, {LD2(s_t + 8 * ns_pad), LD2(s_t + 11 * ns_pad)}));
          const D2 dx = dadd_u({LD2(f), LD2(f + 3 * fs)}, nfx);
          const D2 dy = dadd_u({LD2(f + fs), LD2(f + 4 * fs)}, nfy);
          const D2 dz = dadd_u({LD2(f + 2 * fs), LD2(f + 5 * fs)}, nfz);
#undef LD2
          const D2 rd = dadd_n(dadd_u(dmul_u(rx, dx), dmul_u(ry, dy)), dmul_u(rz, dz));
          const D2 sc = dmul_u(dmul_u(dmul_u(rn, i2), dmul_u(rd, i2)), ir);
          // the accumulators stay normalised: an unnormalised lo would collect
          // rounding errors over ~N/2 additions per lane
          ax = dadd_n(ax, dmul_u(sc, rx));
          ay = dadd_n(ay, dmul_u(sc, ry));
          az = dadd_n(az, dmul_u(sc, rz));
        }
      }
    }
    if (p < N) {
      double* o = partial + ((size_t)slot * N + p) * 3;
      o[0] = ((double)ax.hi.x + (double)ax.hi.y) + ((double)ax.lo.x + (double)ax.lo.y);
      o[1] = ((double)ay.hi.x + (double)ay.hi.y) + ((double)ay.lo.x + (double)ay.lo.y);
      o[2] = ((double)az.hi.x + (double)az.hi.y) + ((double)az.lo.x + (double)az.lo.y);
    }
  }
}

// FP64 stresslet sum, same decomposition, one target per thread.
__global__ void __launch_bounds__(PAIR_THREADS)
k_pair64(int N, int ns, Units un, const double* __restrict__ tmpl64, const double* __restrict__ centers,
         const double* __restrict__ phi, double* __restrict__ partial) {
  extern __shared__ double smd[];
  double* s_t = smd;                       // [ns][6]: xi(3), wn(3)
  double* s_f = s_t + 6 * ns;              // [PAIR_CHUNK][ns][3]
  for (int t = threadIdx.x; t < 6 * ns; t += blockDim.x) s_t[t] = tmpl64[8 * (t / 6) + t % 6];
  const int M = un.M;
  const int c = blockIdx.x;
  int u = un.start(c);
  const int uend = un.start(c + 1);
  while (u < uend) {
    const int tb = u / M, jb0 = u - tb * M;
    const int jb1 = min(M, jb0 + (uend - u));
    const int slot = c - un.first_cta(tb);
    u += jb1 - jb0;
    const int p = tb * blockDim.x + threadIdx.x;
    const int pc = p < N ? p : N - 1;
    const int bi = pc / ns, qi = pc - bi * ns;
    const double xpx = tmpl64[8 * qi], xpy = tmpl64[8 * qi + 1], xpz = tmpl64[8 * qi + 2];
    const double cix = centers[3 * bi], ciy = centers[3 * bi + 1], ciz = centers[3 * bi + 2];
    const double fpx = phi[3 * pc], fpy = phi[3 * pc + 1], fpz = phi[3 * pc + 2];
    double ax = 0.0, ay = 0.0, az = 0.0;
    for (int jc = jb0; jc < jb1; jc += PAIR_CHUNK) {
      const int nb = min(PAIR_CHUNK, jb1 - jc);
      __syncthreads();
      const double* src = phi + 3 * (size_t)jc * ns;
      for (int t = threadIdx.x; t < 3 * nb * ns; t += blockDim.x) s_f[t] = src[t];
      __syncthreads();
      for (int b = 0; b < nb; b++) {
        const int j = jc + b;
        const double ex = (cix - centers[3 * j]) + xpx;
        const double ey = (ciy - centers[3 * j + 1]) + xpy;
        const double ez = (ciz - centers[3 * j + 2]) + xpz;
        const double* fb = s_f + 3 * b * ns;
#pragma unroll 2
        for (int q = 0; q < ns; q++) {
          const double* tq = s_t + 6 * q;
          const double rx = ex - tq[0], ry = ey - tq[1], rz = ez - tq[2];
          const double r2 = fma(rz, rz, fma(ry, ry, fma(rx, rx, EPS64)));
          const double ir = rsqrt(r2);
          const double i2 = ir * ir;
          const double rn = rx * tq[3] + ry * tq[4] + rz * tq[5];
          const double dx = fb[3 * q] - fpx, dy = fb[3 * q + 1] - fpy, dz = fb[3 * q + 2] - fpz;
          const double rd = rx * dx + ry * dy + rz * dz;
          const double s = ((rn * i2) * (rd * i2)) * ir;
          ax = fma(s, rx, ax);
          ay = fma(s, ry, ay);
          az = fma(s, rz, az);
        }
      }
    }
    if (p < N) {
      double* o = partial + ((size_t)slot * N + p) * 3;
      o[0] = ax;
      o[1] = ay;
      o[2] = az;
    }
  }
}

// Rigid coefficients of P phi per body: c = G^{-1} [sum w phi ; sum w xi x phi].
// One warp per body; fixed reduction order.
__global__ void k_moments(int M, int ns, const double* __restrict__ tmpl64, const double* __restrict__ phi,
                          const double* __restrict__ ginv, double* __restrict__ coef) {
  const int body = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (body >= M) return;
  double m[6] = {0, 0, 0, 0, 0, 0};
  for (int q = lane; q < ns; q += 32) {
    const double* o = tmpl64 + 8 * q;
    const double* f = phi + 3 * ((size_t)body * ns + q);
    const double w = o[6];
    m[0] += w * f[0];
    m[1] += w * f[1];
    m[2] += w * f[2];
    m[3] += w * (o[1] * f[2] - o[2] * f[1]);
    m[4] += w * (o[2] * f[0] - o[0] * f[2]);
    m[5] += w * (o[0] * f[1] - o[1] * f[0]);
  }
#pragma unroll
  for (int k = 0; k < 6; k++) m[k] = warp_sum(m[k]);
  if (lane == 0) {
    for (int k = 0; k < 6; k++) {
      double s = 0.0;
      for (int l = 0; l < 6; l++) s += ginv[6 * k + l] * m[l];
      coef[6 * body + k] = s;
    }
  }
}

// out_p = sum over splits of the pair partials + (P phi)_p, (P phi)_p = t_i + w_i x xi_p.
__global__ void k_finish(int N, int ns, int splits, const double* __restrict__ partial,
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
  const double* c = coef + 6 * i;
  const double* xi = tmpl64 + 8 * q;
  a0 += c[0] + (c[4] * xi[2] - c[5] * xi[1]);
  a1 += c[1] + (c[5] * xi[0] - c[3] * xi[2]);
  a2 += c[2] + (c[3] * xi[1] - c[4] * xi[0]);
  out[3 * p] = a0;
  out[3 * p + 1] = a1;
  out[3 * p + 2] = a2;
}

__global__ void k_to_f32(int L, const double* __restrict__ x, float* __restrict__ y) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < L) y[t] = __double2float_rn(x[t]);
}

// rhs_p = s_p - sum_j [G(x_p - c_j) F_j + R(x_p - c_j) T_j]; Stokeslet
// G(r) = (I/|r| + r r^T/|r|^3)/(8 pi mu), rotlet R(r) T = (T x r)/(8 pi mu |r|^3),
// Janus slip s = -(I - n n^T) e on n . e >= 0.
__global__ void k_rhs(int N, int ns, int M, double a, double mu, const double* __restrict__ tmpl64,
                      const double* __restrict__ centers, const double* __restrict__ FT,
                      const double* __restrict__ axes, double* __restrict__ rhs) {
  __shared__ double s_c[128 * 3];
  __shared__ double s_ft[128 * 6];
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  const int pc = p < N ? p : N - 1;
  const int i = pc / ns, q = pc % ns;
  const double* xi = tmpl64 + 8 * q;
  const double cix = centers[3 * i], ciy = centers[3 * i + 1], ciz = centers[3 * i + 2];
  double u0 = 0.0, u1 = 0.0, u2 = 0.0;
  const double k = 1.0 / (8.0 * LCP_PI * mu);
  for (int j0 = 0; j0 < M; j0 += 128) {
    const int nb = min(128, M - j0);
    __syncthreads();
    for (int t = threadIdx.x; t < 3 * nb; t += blockDim.x) s_c[t] = centers[3 * j0 + t];
    for (int t = threadIdx.x; t < 6 * nb; t += blockDim.x) s_ft[t] = FT[6 * j0 + t];
    __syncthreads();
    for (int b = 0; b < nb; b++) {
      const double rx = (cix - s_c[3 * b]) + xi[0];
      const double ry = (ciy - s_c[3 * b + 1]) + xi[1];
      const double rz = (ciz - s_c[3 * b + 2]) + xi[2];
      const double r2 = rx * rx + ry * ry + rz * rz;
      const double ir = 1.0 / sqrt(r2);
      const double ir3 = ir * ir * ir;
      const double* f = s_ft + 6 * b;
      const double rF = rx * f[0] + ry * f[1] + rz * f[2];
      u0 += k * (f[0] * ir + rx * rF * ir3) + k * (f[4] * rz - f[5] * ry) * ir3;
      u1 += k * (f[1] * ir + ry * rF * ir3) + k * (f[5] * rx - f[3] * rz) * ir3;
      u2 += k * (f[2] * ir + rz * rF * ir3) + k * (f[3] * ry - f[4] * rx) * ir3;
    }
  }
  if (p >= N) return;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0;
  if (axes) {
    const double nx = xi[0] / a, ny = xi[1] / a, nz = xi[2] / a;
    const double ex = axes[3 * i], ey = axes[3 * i + 1], ez = axes[3 * i + 2];
    const double ne = nx * ex + ny * ey + nz * ez;
    if (ne >= 0.0) {
      s0 = -(ex - ne * nx);
      s1 = -(ey - ne * ny);
      s2 = -(ez - ne * nz);
    }
  }
  rhs[3 * p] = s0 - u0;
  rhs[3 * p + 1] = s1 - u1;
  rhs[3 * p + 2] = s2 - u2;
}

// The same right-hand side in double-FP32 arithmetic (mixed-precision mode):
// two targets per thread in the lanes of packed double-float values; every
// sum and product is an error-free transformation (TwoSum, TwoProd by FMA),
// |r|^-1 is the special-function seed refined by one Newton step in
// double-float, so each term carries ~2^-44 relative error, on the FP32 pipe
// (64x the FP64 rate).  Stokeslet and rotlet strengths are pre-scaled by
// 1/(8 pi mu) in FP64 before the split.
constexpr int RHS_THREADS = 128;
__device__ __forceinline__ float rsqrt_seed(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ D2 dneg(D2 a) { return {neg2(a.hi), neg2(a.lo)}; }
__device__ __forceinline__ D2 ddup(float2 v) { return {f2(v.x), f2(v.y)}; }

__global__ void __launch_bounds__(RHS_THREADS) k_rhs_df(int N, int ns, int M, double a, double mu,
                                                        const double* __restrict__ tmpl64,
                                                        const double* __restrict__ centers,
                                                        const double* __restrict__ FT,
                                                        const double* __restrict__ axes, double* __restrict__ rhs) {
  __shared__ float2 s_c[RHS_THREADS * 3];    // (hi, lo) of every centre component
  __shared__ float2 s_ft[RHS_THREADS * 6];   // (hi, lo) of F / (8 pi mu), T / (8 pi mu)
  const int t0 = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
  int pc[2], bi[2], qi[2];
#pragma unroll
  for (int u = 0; u < 2; u++) {
    pc[u] = min(t0 + u, N - 1);
    bi[u] = pc[u] / ns;
    qi[u] = pc[u] - bi[u] * ns;
  }
  // target positions x_p = c_i + xi_q in double-float, the two targets in the lanes
  D2 X[3];
#pragma unroll
  for (int d = 0; d < 3; d++) {
    const dfl c0 = df_split(centers[3 * bi[0] + d]), c1 = df_split(centers[3 * bi[1] + d]);
    const dfl x0 = df_split(tmpl64[8 * qi[0] + d]), x1 = df_split(tmpl64[8 * qi[1] + d]);
    X[d] = dadd_n({make_float2(c0.hi, c1.hi), make_float2(c0.lo, c1.lo)},
                  {make_float2(x0.hi, x1.hi), make_float2(x0.lo, x1.lo)});
  }
  const double k = 1.0 / (8.0 * LCP_PI * mu);
  D2 U[3] = {{f2(0.f), f2(0.f)}, {f2(0.f), f2(0.f)}, {f2(0.f), f2(0.f)}};
  for (int j0 = 0; j0 < M; j0 += RHS_THREADS) {
    const int nb = min(RHS_THREADS, M - j0);
    __syncthreads();
    for (int t = threadIdx.x; t < 3 * nb; t += blockDim.x) {
      const dfl v = df_split(centers[3 * j0 + t]);
      s_c[t] = make_float2(v.hi, v.lo);
    }
    for (int t = threadIdx.x; t < 6 * nb; t += blockDim.x) {
      const dfl v = df_split(k * FT[6 * j0 + t]);
      s_ft[t] = make_float2(v.hi, v.lo);
    }
    __syncthreads();
    for (int b = 0; b < nb; b++) {
      D2 R[3], F[3], T[3];
#pragma unroll
      for (int d = 0; d < 3; d++) {
        R[d] = dadd_n(X[d], dneg(ddup(s_c[3 * b + d])));
        F[d] = ddup(s_ft[6 * b + d]);
        T[d] = ddup(s_ft[6 * b + 3 + d]);
      }
      const D2 r2 = dadd_u(dadd_u(dsq_u(R[0]), dsq_u(R[1])), dsq_u(R[2]));
      // |r|^-1: seed, then one Newton step y = y0 + y0 (1 - r2 y0^2) / 2 in double-float
      const float2 y0 = make_float2(rsqrt_seed(r2.hi.x), rsqrt_seed(r2.hi.y));
      const float2 yy = mul2(y0, y0);
      const D2 tt = dmul_u(r2, {yy, fma2(y0, y0, neg2(yy))});
      const float2 hh = sub2(sub2(f2(1.f), tt.hi), tt.lo);
      const D2 ir = fast2sum2(y0, mul2(mul2(f2(0.5f), y0), hh));
      const D2 ir3 = dmul_u(dsq_u(ir), ir);
      const D2 rF = dadd_n(dadd_u(dmul_u(R[0], F[0]), dmul_u(R[1], F[1])), dmul_u(R[2], F[2]));
      const D2 s = dmul_u(rF, ir3);
      const D2 cx[3] = {dadd_u(dmul_u(T[1], R[2]), dneg(dmul_u(T[2], R[1]))),
                        dadd_u(dmul_u(T[2], R[0]), dneg(dmul_u(T[0], R[2]))),
                        dadd_u(dmul_u(T[0], R[1]), dneg(dmul_u(T[1], R[0])))};
#pragma unroll
      for (int d = 0; d < 3; d++) {
        const D2 term = dadd_u(dadd_u(dmul_u(F[d], ir), dmul_u(R[d], s)), dmul_u(cx[d], ir3));
        U[d] = dadd_n(U[d], term);
      }
    }
  }
#pragma unroll
  for (int u = 0; u < 2; u++) {
    const int p = t0 + u;
    if (p >= N) continue;
    const double* xi = tmpl64 + 8 * qi[u];
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    if (axes) {
      const int i = bi[u];
      const double nx = xi[0] / a, ny = xi[1] / a, nz = xi[2] / a;
      const double ex = axes[3 * i], ey = axes[3 * i + 1], ez = axes[3 * i + 2];
      const double ne = nx * ex + ny * ey + nz * ez;
      if (ne >= 0.0) {
        s0 = -(ex - ne * nx);
        s1 = -(ey - ne * ny);
        s2 = -(ez - ne * nz);
      }
    }
    const double u0 = u ? (double)U[0].hi.y + (double)U[0].lo.y : (double)U[0].hi.x + (double)U[0].lo.x;
    const double u1 = u ? (double)U[1].hi.y + (double)U[1].lo.y : (double)U[1].hi.x + (double)U[1].lo.x;
    const double u2 = u ? (double)U[2].hi.y + (double)U[2].lo.y : (double)U[2].hi.x + (double)U[2].lo.x;
    rhs[3 * p] = s0 - u0;
    rhs[3 * p + 1] = s1 - u1;
    rhs[3 * p + 2] = s2 - u2;
  }
}

__global__ void k_neg(int L, const double* __restrict__ x, double* __restrict__ y) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < L) y[t] = -x[t];
}

// ------------------------------------------------------------------ host side
size_t stokes_pair_smem(int ns, int precision);
int stokes_sym_apply(lcp_ctx* ctx, double* out);
int stokes_sym_df_apply(lcp_ctx* ctx, double* out);
// One full wave of CTAs for a pair kernel: SMs x resident CTAs per SM, capped
// by the number of (target block, source body) units.
static int pair_targets(int precision, int v32) {
  return precision == LCP_MIXED ? kPair32Variants[v32].tpt * PAIR_THREADS : PAIR_THREADS;
}

static size_t pair32_smem(int ns, int v32) {
  const int ns_pad = (ns + 3) & ~3;
  return sizeof(float) * (6 * ns_pad + 3 * kPair32Variants[v32].chunk * ns_pad);
}

static int pair_grid_v(const lcp_ctx* ctx, int precision, int v32) {
  const int tpb = pair_targets(precision, v32);
  const int units = ((ctx->N + tpb - 1) / tpb) * ctx->M;
  const int per_sm = precision == LCP_MIXED ? ctx->occ32v[v32] : (precision == LCP_DF64 ? ctx->occdf : ctx->occ64);
  int g = ctx->num_sms * (per_sm > 0 ? per_sm : 1);
  return g < units ? g : units;
}

static int pair_grid(const lcp_ctx* ctx, int precision) { return pair_grid_v(ctx, precision, ctx->v32); }

// Largest number of CTAs that touch one target block (partial slots needed).
static int pair_slots_v(const lcp_ctx* ctx, int grid, int precision, int v32) {
  const int tpb = pair_targets(precision, v32);
  const long long units = (long long)((ctx->N + tpb - 1) / tpb) * ctx->M;
  const long long per = units / grid;   // every CTA holds per or per + 1 units
  const long long s = (ctx->M + per - 1) / (per > 0 ? per : 1) + 1;
  return (int)(s < grid ? s : grid);
}

int stokes_coefs(lcp_ctx* ctx, const double* phi, double* coef) {
  const int threads = 128;
  const int blocks = (ctx->M * 32 + threads - 1) / threads;
  ++ctx->nlaunch, k_moments<<<blocks, threads, 0, ctx->stream>>>(ctx->M, ctx->ns, ctx->tmpl64, phi, ctx->ginv, coef);
  LCP_CUDA(cudaGetLastError());
  return LCP_OK;
}

static int stokes_apply_sums(lcp_ctx* ctx, const double* phi, double* out, int precision);

// (K + P) phi with the pair sums of `precision`, plus the self-interaction
// correction of every body when cfg.self_quadrature is on.
int stokes_apply(lcp_ctx* ctx, const double* phi, double* out, int precision) {
  LCP_TRY(stokes_apply_sums(ctx, phi, out, precision));
  if (ctx->cself32) LCP_TRY(self_correction_apply(ctx, phi, out, precision));
  return LCP_OK;
}

static int stokes_apply_sums(lcp_ctx* ctx, const double* phi, double* out, int precision) {
  const int N = ctx->N, ns = ctx->ns, M = ctx->M;
  const int tpb = pair_targets(precision, ctx->v32);
  const int ntb = (N + tpb - 1) / tpb;
  const int grid = pair_grid(ctx, precision);
  const int slots = pair_slots_v(ctx, grid, precision, ctx->v32);
  if (slots > ctx->splits) {
    ctx->err = "internal: pair-sum slots exceed the partial buffer";
    return LCP_ERR_INVALID_ARG;
  }
  Units un{ntb * M, grid, M};
  LCP_TRY(stokes_coefs(ctx, phi, ctx->coef));
  if (precision == LCP_MIXED && ctx->sym) {
    ++ctx->nlaunch, k_to_f32<<<(3 * N + 255) / 256, 256, 0, ctx->stream>>>(3 * N, phi, ctx->phi32);
    ctx->c_fp32++;
    return stokes_sym_apply(ctx, out);
  }
  if (precision == LCP_DF64 && ctx->sym && ctx->symdf_grid > 0 && ctx->symdf_slots <= ctx->splits) {
    ++ctx->nlaunch, k_split_df<<<(3 * N + 255) / 256, 256, 0, ctx->stream>>>(3 * N, phi, ctx->phidf);
    ctx->c_df64++;
    return stokes_sym_df_apply(ctx, out);
  }
  LCP_CUDA(cudaMemsetAsync(ctx->partial, 0, sizeof(double) * 3 * (size_t)N * slots, ctx->stream));
  cudaEvent_t e0 = nullptr;
  if (precision == LCP_MIXED) {
    ++ctx->nlaunch, k_to_f32<<<(3 * N + 255) / 256, 256, 0, ctx->stream>>>(3 * N, phi, ctx->phi32);
    const int ns_pad = (ns + 3) & ~3;
    const size_t smem = pair32_smem(ns, ctx->v32);
    e0 = prof_begin(ctx);
    ++ctx->nlaunch, kPair32Variants[ctx->v32].kernel<<<grid, PAIR_THREADS, smem, ctx->stream>>>(
                        N, ns, ns_pad, un, ctx->tmpl32, ctx->centers32, ctx->phi32, ctx->partial);
    prof_end(ctx, e0, 0);
    ctx->c_fp32++;
  } else if (precision == LCP_DF64) {
    ++ctx->nlaunch, k_split_df<<<(3 * N + 255) / 256, 256, 0, ctx->stream>>>(3 * N, phi, ctx->phidf);
    const int ns_pad = (ns + 3) & ~3;
    const size_t smem = stokes_pair_smem(ns, LCP_DF64);
    e0 = prof_begin(ctx);
    ++ctx->nlaunch, k_pair_df<<<grid, PAIR_THREADS, smem, ctx->stream>>>(N, ns, ns_pad, un, ctx->tmpl64,
                                                                         ctx->centers, ctx->phidf, ctx->partial);
    prof_end(ctx, e0, 2);
    ctx->c_df64++;
  } else {
    const size_t smem = sizeof(double) * (6 * ns + 3 * PAIR_CHUNK * ns);
    e0 = prof_begin(ctx);
    ++ctx->nlaunch, k_pair64<<<grid, PAIR_THREADS, smem, ctx->stream>>>(N, ns, un, ctx->tmpl64, ctx->centers,
                                                                        phi, ctx->partial);
    prof_end(ctx, e0, 1);
    ctx->c_fp64++;
  }
  ++ctx->nlaunch, k_finish<<<(N + 255) / 256, 256, 0, ctx->stream>>>(N, ns, slots, ctx->partial, ctx->coef,
                                                                     ctx->tmpl64, out);
  LCP_CUDA(cudaGetLastError());
  return LCP_OK;
}

// FP64 mode: the FP64 kernel; mixed mode: the double-float kernel (same
// accuracy class, ~2^-44 per operation, on the FP32 pipe).
int stokes_rhs(lcp_ctx* ctx, const double* FT, int include_slip, double* rhs) {
  const int N = ctx->N;
  const double* ax = include_slip && ctx->has_axes ? ctx->axes : nullptr;
  if (ctx->cfg.precision == LCP_FP64)
    ++ctx->nlaunch, k_rhs<<<(N + 127) / 128, 128, 0, ctx->stream>>>(N, ctx->ns, ctx->M, ctx->cfg.radius,
                                                                    ctx->cfg.viscosity, ctx->tmpl64, ctx->centers,
                                                                    FT, ax, rhs);
  else
    ++ctx->nlaunch, k_rhs_df<<<(N + 2 * RHS_THREADS - 1) / (2 * RHS_THREADS), RHS_THREADS, 0, ctx->stream>>>(
                        N, ctx->ns, ctx->M, ctx->cfg.radius, ctx->cfg.viscosity, ctx->tmpl64, ctx->centers, FT, ax,
                        rhs);
  LCP_CUDA(cudaGetLastError());
  return LCP_OK;
}

int stokes_velocity(lcp_ctx* ctx, const double* phi, double* UO) {
  LCP_TRY(stokes_coefs(ctx, phi, ctx->coef));
  ++ctx->nlaunch, k_neg<<<(6 * ctx->M + 127) / 128, 128, 0, ctx->stream>>>(6 * ctx->M, ctx->coef, UO);
  LCP_CUDA(cudaGetLastError());
  return LCP_OK;
}

// Partial slots to allocate: the larger of the two kernels' needs.
int stokes_max_splits(const lcp_ctx* ctx) {
  int m = 0;
  for (int v = 0; v < kNumPair32Variants; v++) {
    const int s = pair_slots_v(ctx, pair_grid_v(ctx, LCP_MIXED, v), LCP_MIXED, v);
    if (s > m) m = s;
  }
  const int precs[2] = {LCP_FP64, LCP_DF64};
  for (int prec : precs) {
    const int s = pair_slots_v(ctx, pair_grid_v(ctx, prec, 0), prec, 0);
    if (s > m) m = s;
  }
  return m;
}

size_t stokes_pair_smem(int ns, int precision) {
  const int ns_pad = (ns + 3) & ~3;
  if (precision == LCP_DF64) return sizeof(float) * (12 * ns_pad + 6 * PAIR_CHUNK * ns_pad);
  return precision == LCP_MIXED ? pair32_smem(ns, 0) : sizeof(double) * (6 * ns + 3 * PAIR_CHUNK * ns);
}

// Shared-memory limits and one-wave grid sizes (occupancy) of the pair kernels.
int stokes_configure(lcp_ctx* ctx) {
  const size_t s64 = stokes_pair_smem(ctx->ns, LCP_FP64);
  if (s64 > 48 * 1024) LCP_CUDA(raise_smem_limit((const void*)k_pair64, s64));
  for (int v = 0; v < kNumPair32Variants; v++) {
    const size_t sv = pair32_smem(ctx->ns, v);
    if (sv > 48 * 1024)
      LCP_CUDA(raise_smem_limit((const void*)kPair32Variants[v].kernel, sv));
    LCP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ctx->occ32v[v], kPair32Variants[v].kernel, PAIR_THREADS, sv));
  }
  int dev = 0;
  LCP_CUDA(cudaGetDevice(&dev));
  LCP_CUDA(cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, dev));
  LCP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ctx->occ64, k_pair64, PAIR_THREADS, s64));
  const size_t sdf = stokes_pair_smem(ctx->ns, LCP_DF64);
  if (sdf > 48 * 1024) LCP_CUDA(raise_smem_limit((const void*)k_pair_df, sdf));
  LCP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ctx->occdf, k_pair_df, PAIR_THREADS, sdf));
  return LCP_OK;
}

// ---------------------------------------------------------------- autotuner
// Chooses the FP32 pair-kernel variant (targets per CTA = target-block size,
// source bodies per shared-memory tile, or the symmetric kernel) for a size
// class by timing every candidate on this context's geometry; the choice is
// cached per (nodes per sphere, bodies) class for the process.
#include <map>
#include <mutex>

static std::mutex g_tune_mu;
static std::map<std::pair<int, int>, int> g_tune_cache;

static int size_class(int M) {   // bodies rounded up to a power of two
  int c = 1;
  while (c < M) c <<= 1;
  return c;
}

int stokes_sym_variant_count();
const char* stokes_sym_variant_name(int v);
bool stokes_sym_variant_usable(const lcp_ctx* ctx, int v);

// Candidate index: plain variants 0 .. kNumPair32Variants-1, then the
// symmetric variants.
static int candidate_count() { return kNumPair32Variants + stokes_sym_variant_count(); }
static void set_candidate(lcp_ctx* ctx, int v) {
  ctx->sym = v >= kNumPair32Variants;
  ctx->v32 = ctx->sym ? 0 : v;
  ctx->sym_v = ctx->sym ? v - kNumPair32Variants : 0;
}
static bool candidate_usable(lcp_ctx* ctx, int v) {
  if (v >= kNumPair32Variants) return stokes_sym_variant_usable(ctx, v - kNumPair32Variants);
  return ctx->occ32v[v] > 0 && pair_slots_v(ctx, pair_grid_v(ctx, LCP_MIXED, v), LCP_MIXED, v) <= ctx->splits;
}
static const char* candidate_name(int v) {
  return v >= kNumPair32Variants ? stokes_sym_variant_name(v - kNumPair32Variants) : kPair32Variants[v].name;
}

int stokes_autotune(lcp_ctx* ctx) {
  const std::pair<int, int> key(ctx->ns, size_class(ctx->M));
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune_cache.find(key);
    // a size class spans a factor of two in bodies: the cached choice is taken
    // only where it also fits this context (slots, or no symmetric buffers)
    if (it != g_tune_cache.end() && candidate_usable(ctx, it->second)) {
      set_candidate(ctx, it->second);
      return LCP_OK;
    }
  }
  const int L = 3 * ctx->N;
  // a deterministic density: phi = sin(k) pattern, built on the device
  double* phi = ctx->dphi;
  double* out = ctx->wv;
  std::vector<double> h(L);
  for (int i = 0; i < L; i++) h[i] = std::sin(0.37 * i);
  LCP_CUDA(cudaMemcpyAsync(phi, h.data(), sizeof(double) * L, cudaMemcpyHostToDevice, ctx->stream));
  cudaEvent_t a, b;
  LCP_CUDA(cudaEventCreate(&a));
  LCP_CUDA(cudaEventCreate(&b));
  float best = 1e30f;
  int best_v = 0;
  const bool prof = ctx->prof;
  ctx->prof = false;
  for (int v = 0; v < candidate_count(); v++) {
    if (!candidate_usable(ctx, v)) continue;
    set_candidate(ctx, v);
    LCP_TRY(stokes_apply(ctx, phi, out, LCP_MIXED));   // warm-up
    LCP_CUDA(cudaEventRecord(a, ctx->stream));
    for (int r = 0; r < 3; r++) LCP_TRY(stokes_apply(ctx, phi, out, LCP_MIXED));
    LCP_CUDA(cudaEventRecord(b, ctx->stream));
    LCP_CUDA(cudaEventSynchronize(b));
    float ms = 0.f;
    LCP_CUDA(cudaEventElapsedTime(&ms, a, b));
    if (ms < best) { best = ms; best_v = v; }
  }
  ctx->prof = prof;
  ctx->c_fp32 = 0;
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  set_candidate(ctx, best_v);
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune_cache[key] = best_v;
  return LCP_OK;
}

const char* stokes_variant_name(const lcp_ctx* ctx) {
  return candidate_name(ctx->sym ? kNumPair32Variants + ctx->sym_v : ctx->v32);
}

// Forces a variant by name (LCP_ERR_INVALID_ARG if unknown or unusable here).
int stokes_select_variant(lcp_ctx* ctx, const char* name) {
  for (int v = 0; v < candidate_count(); v++)
    if (std::strcmp(candidate_name(v), name) == 0) {
      if (!candidate_usable(ctx, v)) break;
      set_candidate(ctx, v);
      return LCP_OK;
    }
  ctx->err = std::string("kernel variant not available: ") + name;
  return LCP_ERR_INVALID_ARG;
}
