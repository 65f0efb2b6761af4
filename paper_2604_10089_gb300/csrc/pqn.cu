// Proximal quasi-Newton kernels (Sec. 4 and 5 of the paper).
//
//  * Algorithm 1 (Mono-PQN): x_tilde = x - H g, with H the inverse of the
//    unrolled BFGS model B = delta I + U U^T - V V^T (Appendix D.1; B_0 =
//    delta I scaled by the first secant pair, or I), applied by the Woodbury
//    identity on [U V] (the same H as the two-loop recursion over the stored
//    pairs), x_hat = prox^B(x_tilde), p = x_hat - x, one MVP A[p], the optimal
//    over-relaxation of Algorithm 2, x += eta p, g += eta A[p] (MVP reuse),
//    BFGS update with s = eta p, y = eta A[p].
//  * Proposition 1 / Appendix A.2: the weighted prox by semi-smooth Newton on
//    G(a, at) = [a + U^T(xt + C^-1 V at - z); at + V^T(xt - z)],
//    z = (xt + C^-1 V at - U a / delta)_+, C = delta I + U U^T, with the generalised
//    Jacobian J = I + [U^T L U, U^T (I - L) C^-1 V; V^T L U, -V^T L C^-1 V],
//    L = diag(z > 0).  G and z are FP64; J is assembled and factorised in
//    FP32 (an inexact Jacobian only changes the Newton path, not the root).
//  * Algorithm 4 (Bi-PQN): the outer update of x, g and of the high-fidelity
//    corrections U_h, V_h (B^(k+1) = B^(k) + u u^T - v v^T with
//    B^(k) s = eta (A_hat x_hat - A_hat x) + U_h U_h^T s - V_h V_h^T s,
//    Appendix D.2) and the secant carry-over Y_low <- Y_hat + (u u^T - v v^T) S_hat.
//
// The n-vectors are small (one entry per contact), so each phase runs in a
// single thread block; the MVPs in between use the whole GPU.
#include <algorithm>
#include <cmath>

#include "common.cuh"

namespace {
constexpr int PQN_T = 512;
constexpr int PQN_W = PQN_T / 32;
}

// scal slots of a PqnDev
enum {
  S_KKT = 0, S_KKTDOT = 1, S_FLAG = 2, S_ETA = 3, S_SSN_IT = 4, S_SSN_FAIL = 5, S_PG = 6, S_PAP = 7,
  S_ACCEPT = 8, S_BLK = 9, S_TAU = 10, S_DELTA = 11, S_DSET = 12, S_NSCAL = 16
};

// Per-run workspace laid out after the PqnDev vectors (device pointers).
struct PqnWork {
  double *y, *z, *d, *q;    // [n]
  float *U32, *V32;         // [rmax][n]
  float* lam;               // [n]
  double* ys;               // [rmax] y^T s per pair
};

__device__ __forceinline__ double bsum(double v, double* red) { return block_sum(v, red); }

// Scale of the initial model B_0 = delta I (H_0 = I / delta); 1 until set.
__device__ __forceinline__ double delta_of(const PqnDev& pq) {
  return pq.scal[S_DSET] != 0.0 ? pq.scal[S_DELTA] : 1.0;
}

// out[k] = M[k] . v for k < rows (warp per row, fixed lane order).  out in smem or global.
__device__ void bmultidot(const double* __restrict__ Mt, int n, int rows, const double* __restrict__ v,
                          double* out) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int k = w; k < rows; k += PQN_W) {
    const double* m = Mt + (size_t)k * n;
    double s = 0.0;
    for (int i = lane; i < n; i += 32) s += m[i] * v[i];
    s = warp_sum(s);
    if (lane == 0) out[k] = s;
  }
  __syncthreads();
}

// Solves A X = B (A: m x m row-major, leading dimension lda; B: m x nr) by
// Gaussian elimination with partial pivoting, block-parallel.  Rows are not
// exchanged: step k takes the unused row with the largest |A[i][k]| (warp 0),
// then all threads eliminate column k from the other unused rows (two block
// barriers per step).  Back substitution runs one warp per right-hand side.
// X (m x nr, leading dimension ldx) receives the solution; A and B are
// overwritten.  perm, used: int[m] in shared memory.  T = double or float.
template <typename T>
__device__ void pivot_solve(T* A, int lda, T* B, int ldb, int m, int nr, T* X, int ldx, int* perm, int* used) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = threadIdx.x; i < m; i += blockDim.x) used[i] = 0;
  __syncthreads();
  for (int k = 0; k < m; k++) {
    if (w == 0) {
      T best = T(-1);
      int arg = m;
      for (int i = lane; i < m; i += 32)
        if (!used[i]) {
          const T v = fabs(A[i * lda + k]);
          if (v > best) { best = v; arg = i; }
        }
      for (int o = 16; o > 0; o >>= 1) {
        const T ov = __shfl_xor_sync(0xffffffffu, best, o);
        const int oa = __shfl_xor_sync(0xffffffffu, arg, o);
        if (ov > best || (ov == best && oa < arg)) { best = ov; arg = oa; }
      }
      if (lane == 0) { perm[k] = arg; used[arg] = 1; }
    }
    __syncthreads();
    const int p = perm[k];
    const T piv = A[p * lda + k];
    const int ca = m - k - 1, cols = ca + nr;
    for (int t = threadIdx.x; t < m * cols; t += blockDim.x) {
      const int i = t / cols, c = t - i * cols;
      if (used[i]) continue;
      const T f = A[i * lda + k] / piv;
      if (c < ca) A[i * lda + k + 1 + c] -= f * A[p * lda + k + 1 + c];
      else B[i * ldb + (c - ca)] -= f * B[p * ldb + (c - ca)];
    }
    __syncthreads();
  }
  for (int c = w; c < nr; c += nw) {
    for (int k = m - 1; k >= 0; k--) {
      const int p = perm[k];
      const T xk = B[p * ldb + c] / A[p * lda + k];
      for (int kk = lane; kk < k; kk += 32) {
        const int q = perm[kk];
        B[q * ldb + c] -= A[q * lda + k] * xk;
      }
      if (lane == 0) X[k * ldx + c] = xk;
      __syncwarp();
    }
  }
  __syncthreads();
}

// Shared-memory layout of the direction kernel for r <= R pairs.
constexpr int GRAM_CHUNK = 64;   // contacts staged per chunk of the masked Grams
struct ProxSmem {
  double *X, *UCV, *VCV, *tmp, *XB, *XS, *al, *alt, *G, *Gt, *c, *udv, *wg, *cw;
  float *J, *gf, *dx, *GUU, *GVU, *GVV, *T1, *T2, *Um, *Vm;
  int *perm, *used;
};

__device__ ProxSmem prox_smem(void* base, int R) {
  ProxSmem s;
  double* d = (double*)base;
  s.X = d; d += R * R;
  s.UCV = d; d += R * R;
  s.VCV = d; d += R * R;
  s.tmp = d; d += R * R;
  s.XB = d; d += R * (R + 1);
  s.XS = d; d += R * (R + 1);
  s.al = d; d += 2 * R;
  s.alt = d; d += 2 * R;
  s.G = d; d += 2 * R;
  s.Gt = d; d += 2 * R;
  s.c = d; d += 2 * R;
  s.udv = d; d += 2 * R;
  s.wg = d; d += 2 * R;
  s.cw = d; d += 2 * R;
  float* f = (float*)d;
  s.J = f; f += 4 * R * R;
  s.gf = f; f += 2 * R;
  s.dx = f; f += 2 * R;
  s.GUU = f; f += R * R;
  s.GVU = f; f += R * R;
  s.GVV = f; f += R * R;
  s.T1 = f; f += R * R;
  s.T2 = f; f += R * R;
  const int Re = (R + 1) & ~1;
  s.Um = f; f += Re * (GRAM_CHUNK + 1);
  s.Vm = f; f += Re * (GRAM_CHUNK + 1);
  s.perm = (int*)f;
  s.used = s.perm + 2 * R;
  return s;
}

__host__ __device__ inline size_t prox_smem_bytes(int R) {
  const int Re = (R + 1) & ~1;
  return sizeof(double) * (4 * R * R + 2 * R * (R + 1) + 16 * R) +
         sizeof(float) * (9 * R * R + 4 * R + 2 * Re * (GRAM_CHUNK + 1)) + sizeof(int) * 4 * R + 64;
}

// Masked Grams GUU = U^T L U, GVU = V^T L U, GVV = V^T L V (FP32, r x r,
// row-major), L = diag(lam) with lam in {0, 1}: with Um = L U and Vm = L V
// they are Um^T Um, Vm^T Um, Vm^T Vm.  Contacts are staged through shared
// memory GRAM_CHUNK at a time (row stride GRAM_CHUNK + 1: conflict-free);
// each thread accumulates 2 x 2 blocks, the symmetric Grams only on and
// above the diagonal.
__device__ void masked_grams(const PqnWork& wk, int n, int r, ProxSmem& sm) {
  const int re = (r + 1) & ~1, h = re / 2;
  const int ntri = h * (h + 1) / 2, nblk = 2 * ntri + h * h;
  constexpr int LD = GRAM_CHUNK + 1;
  float acc[2][4];
  for (int q = 0; q < 2; q++)
    for (int e = 0; e < 4; e++) acc[q][e] = 0.f;
  for (int i0 = 0; i0 < n; i0 += GRAM_CHUNK) {
    __syncthreads();
    for (int t = threadIdx.x; t < re * GRAM_CHUNK; t += blockDim.x) {
      const int k = t / GRAM_CHUNK, ii = t - k * GRAM_CHUNK, i = i0 + ii;
      const bool in = k < r && i < n;
      const float l = in ? wk.lam[i] : 0.f;
      sm.Um[k * LD + ii] = in ? l * wk.U32[(size_t)k * n + i] : 0.f;
      sm.Vm[k * LD + ii] = in ? l * wk.V32[(size_t)k * n + i] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 2; q++) {
      const int bidx = threadIdx.x + q * blockDim.x;
      if (bidx >= nblk) break;
      int which, bk, bl;   // 0: UU (bk <= bl), 1: VU, 2: VV (bk <= bl)
      if (bidx < ntri || bidx >= ntri + h * h) {
        which = bidx < ntri ? 0 : 2;
        int t = bidx < ntri ? bidx : bidx - ntri - h * h;
        bk = 0;
        while (t >= h - bk) { t -= h - bk; bk++; }
        bl = bk + t;
      } else {
        which = 1;
        const int t = bidx - ntri;
        bk = t / h;
        bl = t - bk * h;
      }
      const float* A = which == 0 ? sm.Um : sm.Vm;
      const float* B = which == 2 ? sm.Vm : sm.Um;
      const float* a0 = A + (2 * bk) * LD;
      const float* a1 = a0 + LD;
      const float* b0 = B + (2 * bl) * LD;
      const float* b1 = b0 + LD;
      float s00 = acc[q][0], s01 = acc[q][1], s10 = acc[q][2], s11 = acc[q][3];
#pragma unroll 8
      for (int ii = 0; ii < GRAM_CHUNK; ii++) {
        const float x0 = a0[ii], x1 = a1[ii], y0 = b0[ii], y1 = b1[ii];
        s00 = fmaf(x0, y0, s00);
        s01 = fmaf(x0, y1, s01);
        s10 = fmaf(x1, y0, s10);
        s11 = fmaf(x1, y1, s11);
      }
      acc[q][0] = s00; acc[q][1] = s01; acc[q][2] = s10; acc[q][3] = s11;
    }
  }
#pragma unroll
  for (int q = 0; q < 2; q++) {
    const int bidx = threadIdx.x + q * blockDim.x;
    if (bidx >= nblk) break;
    int which, bk, bl;
    if (bidx < ntri || bidx >= ntri + h * h) {
      which = bidx < ntri ? 0 : 2;
      int t = bidx < ntri ? bidx : bidx - ntri - h * h;
      bk = 0;
      while (t >= h - bk) { t -= h - bk; bk++; }
      bl = bk + t;
    } else {
      which = 1;
      const int t = bidx - ntri;
      bk = t / h;
      bl = t - bk * h;
    }
    float* Gm = which == 0 ? sm.GUU : (which == 1 ? sm.GVU : sm.GVV);
    for (int e = 0; e < 4; e++) {
      const int k = 2 * bk + (e >> 1), l = 2 * bl + (e & 1);
      if (k >= r || l >= r) continue;
      Gm[k * r + l] = acc[q][e];
      if (which != 1) Gm[l * r + k] = acc[q][e];
    }
  }
  __syncthreads();
}

// Residual of the prox root function at (al = [a; at]); writes z, the mask
// and G; returns ||G||.
__device__ double ssn_residual(const PqnDev& pq, const PqnWork& wk, int r, const double* xt, const double* al,
                               ProxSmem& sm, double* G, double* red) {
  const int n = pq.n;
  const double* a = al;
  const double* at = al + r;
  // c = X at + a
  for (int k = threadIdx.x; k < r; k += blockDim.x) {
    double s = a[k];
    for (int l = 0; l < r; l++) s += sm.X[k * r + l] * at[l];
    sm.c[k] = s;
  }
  __syncthreads();
  const double idl = 1.0 / delta_of(pq);
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double y = 0.0;
    for (int k = 0; k < r; k++) y += pq.V[(size_t)k * n + i] * at[k] - pq.U[(size_t)k * n + i] * sm.c[k];
    y = xt[i] + idl * y;
    const double z = y > 0.0 ? y : 0.0;
    wk.z[i] = z;
    wk.lam[i] = y > 0.0 ? 1.f : 0.f;
    wk.d[i] = xt[i] - z;
  }
  __syncthreads();
  bmultidot(pq.U, n, r, wk.d, sm.udv);
  bmultidot(pq.V, n, r, wk.d, sm.udv + r);
  for (int k = threadIdx.x; k < r; k += blockDim.x) {
    double s = 0.0;
    for (int l = 0; l < r; l++) s += sm.UCV[k * r + l] * at[l];
    s = a[k] + sm.udv[k] + idl * s;
    G[k] = s;
    G[r + k] = at[k] + sm.udv[r + k];
  }
  __syncthreads();
  double part = 0.0;
  for (int k = threadIdx.x; k < 2 * r; k += blockDim.x) part += G[k] * G[k];
  return sqrt(bsum(part, red));
}

// z = prox^B(xt), B = delta I + U U^T - V V^T with r pairs.  The caller has
// set sm.X = C^-1 U^T V (C = delta I + U^T U), sm.UCV = U^T V - U^T U X and
// sm.VCV = V^T V - V^T U X.  Returns Newton steps (negative when the
// fallback coordinate descent was needed).
__device__ int prox_ssn(const PqnDev& pq, const PqnWork& wk, int r, const double* xt, double* zout,
                        ProxSmem& sm, double* red, int jmax) {
  const int n = pq.n;
  if (r == 0) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) zout[i] = xt[i] > 0.0 ? xt[i] : 0.0;
    __syncthreads();
    return 0;
  }
  for (int k = threadIdx.x; k < 2 * r; k += blockDim.x) sm.al[k] = 0.0;
  __syncthreads();
  double xn = 0.0;
  {
    double part = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) part += xt[i] * xt[i];
    xn = sqrt(bsum(part, red));
  }
  const double scale = 1.0 + xn;
  double gn = ssn_residual(pq, wk, r, xt, sm.al, sm, sm.G, red);
  int j = 0;
  bool ok = false;
  for (; j < jmax; j++) {
    if (gn <= 1e-13 * scale) { ok = true; break; }
    masked_grams(wk, n, r, sm);
    // T1 = GUU X, T2 = GVU X
    for (int t = threadIdx.x; t < r * r; t += blockDim.x) {
      const int k = t / r, l = t % r;
      float s1 = 0.f, s2 = 0.f;
      for (int m = 0; m < r; m++) {
        s1 += sm.GUU[k * r + m] * (float)sm.X[m * r + l];
        s2 += sm.GVU[k * r + m] * (float)sm.X[m * r + l];
      }
      sm.T1[t] = s1;
      sm.T2[t] = s2;
    }
    __syncthreads();
    const int m2 = 2 * r;
    const float jscale = (float)(1.0 / delta_of(pq));
    for (int t = threadIdx.x; t < m2 * m2; t += blockDim.x) {
      const int row = t / m2, col = t % m2;
      float v;
      if (row < r && col < r) v = sm.GUU[row * r + col];
      else if (row < r) {  // U^T (I - L) C^-1 V = UCV - (U^T L V - U^T L U X)
        const int l = col - r;
        v = (float)sm.UCV[row * r + l] - (sm.GVU[l * r + row] - sm.T1[row * r + l]);
      } else if (col < r) v = sm.GVU[(row - r) * r + col];
      else {  // -V^T L C^-1 V = -(V^T L V - V^T L U X)
        const int k = row - r, l = col - r;
        v = -(sm.GVV[k * r + l] - sm.T2[k * r + l]);
      }
      sm.J[t] = v * jscale + (row == col ? 1.f : 0.f);
    }
    for (int k = threadIdx.x; k < m2; k += blockDim.x) sm.gf[k] = (float)sm.G[k];
    __syncthreads();
    pivot_solve<float>(sm.J, m2, sm.gf, 1, m2, 1, sm.dx, 1, sm.perm, sm.used);
    // backtracking on ||G||
    double t = 1.0;
    for (int bt = 0; bt < 30; bt++) {
      for (int k = threadIdx.x; k < m2; k += blockDim.x) sm.alt[k] = sm.al[k] - t * (double)sm.dx[k];
      __syncthreads();
      const double gt = ssn_residual(pq, wk, r, xt, sm.alt, sm, sm.Gt, red);
      if (gt <= (1.0 - 1e-4 * t) * gn || t < 1e-8) {
        gn = gt;
        break;
      }
      t *= 0.5;
    }
    for (int k = threadIdx.x; k < m2; k += blockDim.x) {
      sm.al[k] = sm.alt[k];
      sm.G[k] = sm.Gt[k];
    }
    __syncthreads();
  }
  if (ok || gn <= 1e-9 * scale) {
    // z of the accepted iterate is in wk.z
    for (int i = threadIdx.x; i < n; i += blockDim.x) zout[i] = wk.z[i];
    __syncthreads();
    return j;
  }
  // Fallback: projected Gauss-Seidel on min_{z>=0} 1/2 (z - xt)^T B (z - xt),
  // B applied through a = U^T (z - xt), b = V^T (z - xt) (warp 0 only).
  for (int i = threadIdx.x; i < n; i += blockDim.x) { zout[i] = xt[i] > 0.0 ? xt[i] : 0.0; wk.d[i] = zout[i] - xt[i]; }
  __syncthreads();
  bmultidot(pq.U, n, r, wk.d, sm.udv);
  bmultidot(pq.V, n, r, wk.d, sm.udv + r);
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    // bounded: a model that needs more sweeps is far from convex (e.g. a low-fidelity
    // operator that is not positive definite); the best iterate is returned
    for (int sweep = 0; sweep < 400; sweep++) {
      double worst = 0.0;
      for (int l = 0; l < n; l++) {
        double gr = 0.0, bll = 0.0;
        for (int k = lane; k < r; k += 32) {
          const double u = pq.U[(size_t)k * n + l], v = pq.V[(size_t)k * n + l];
          gr += u * sm.udv[k] - v * sm.udv[r + k];
          bll += u * u - v * v;
        }
        gr = warp_sum(gr);
        bll = warp_sum(bll);
        gr += delta_of(pq) * (zout[l] - xt[l]);
        bll += delta_of(pq);
        const double zn = fmax(0.0, zout[l] - gr / bll);
        const double dz = zn - zout[l];
        const double kk = fabs(fmin(zout[l], gr));
        worst = fmax(worst, kk);
        __syncwarp();
        if (lane == 0) zout[l] = zn;
        for (int k = lane; k < r; k += 32) {
          sm.udv[k] += dz * pq.U[(size_t)k * n + l];
          sm.udv[r + k] += dz * pq.V[(size_t)k * n + l];
        }
        __syncwarp();
      }
      if (worst <= 1e-14 * scale) break;
    }
  }
  __syncthreads();
  return -jmax;
}

// --------------------------------------------------------------- kernels

// x = max(x0, 0) (or 0); the caller follows with an MVP and k_pqn_grad.
__global__ void __launch_bounds__(PQN_T) k_pqn_init(PqnDev pq, const double* x0) {
  for (int i = threadIdx.x; i < pq.n; i += blockDim.x) pq.x[i] = x0 ? fmax(x0[i], 0.0) : 0.0;
  for (int i = threadIdx.x; i < pq.n; i += blockDim.x) pq.extra[i] = 0.0;
}

// g = Ax + b (or g = g0); kkt = ||min(x, g)||_2, kkt_dot = <x, g>.
__global__ void __launch_bounds__(PQN_T) k_pqn_grad(PqnDev pq, const double* Ax, const double* b, const double* g0) {
  __shared__ double red[32];
  double p1 = 0.0, p2 = 0.0;
  for (int i = threadIdx.x; i < pq.n; i += blockDim.x) {
    const double g = g0 ? g0[i] : Ax[i] + b[i];
    pq.g[i] = g;
    const double m = fmin(pq.x[i], g);
    p1 += m * m;
    p2 += pq.x[i] * g;
  }
  const double k1 = block_sum(p1, red);
  const double k2 = block_sum(p2, red);
  if (threadIdx.x == 0) {
    pq.scal[S_KKT] = sqrt(k1);
    pq.scal[S_KKTDOT] = k2;
  }
}

// Direction of Algorithm 1: xt = x - H g, xh = prox^B(xt), p = xh - x, with
// the projected-gradient fallback when p^T g >= 0 (memory reset).  H g is
// taken from the unrolled model B = delta I + W S W^T (W = [U V],
// S = diag(I, -I)) by the Woodbury identity,
//   H g = (g - W K^-1 W^T g) / delta,   K = delta S + W^T W,
// with K eliminated in blocks through C = delta I + U^T U (whose solve with
// U^T V the prox needs as well) and the Schur complement
// V^T V - V^T U C^-1 U^T V - delta I; this is the same H as the two-loop
// recursion over the stored pairs, in O(n r + r^3) work without a chain of
// 2r reductions.
__global__ void __launch_bounds__(PQN_T) k_pqn_direction(PqnDev pq, PqnWork wk, int jmax) {
  extern __shared__ double smem[];
  __shared__ double red[32];
  const int n = pq.n;
  const int r = *pq.r;
  const int R = pq.rmax;
  const double dl = delta_of(pq), idl = 1.0 / dl;
  ProxSmem sm = prox_smem(smem, R);
  if (r == 0) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) pq.xt[i] = pq.x[i] - idl * pq.g[i];
    __syncthreads();
  } else {
    bmultidot(pq.U, n, r, pq.g, sm.wg);       // U^T g
    bmultidot(pq.V, n, r, pq.g, sm.wg + r);   // V^T g
    // C [X | y1] = [U^T V | U^T g]
    for (int t = threadIdx.x; t < r * r; t += blockDim.x) {
      const int k = t / r, l = t - k * r;
      sm.tmp[t] = pq.UU[k * R + l] + (k == l ? dl : 0.0);
    }
    for (int t = threadIdx.x; t < r * (r + 1); t += blockDim.x) {
      const int k = t / (r + 1), l = t - k * (r + 1);
      sm.XB[t] = l < r ? pq.UV[k * R + l] : sm.wg[k];
    }
    __syncthreads();
    pivot_solve<double>(sm.tmp, r, sm.XB, r + 1, r, r + 1, sm.XS, r + 1, sm.perm, sm.used);
    for (int t = threadIdx.x; t < r * r; t += blockDim.x) {
      const int k = t / r, l = t - k * r;
      sm.X[t] = sm.XS[k * (r + 1) + l];
    }
    __syncthreads();
    // UCV = UV - UU X ; VCV = VV - UV^T X
    for (int t = threadIdx.x; t < r * r; t += blockDim.x) {
      const int k = t / r, l = t % r;
      double s1 = pq.UV[k * R + l], s2 = pq.VV[k * R + l];
      for (int m = 0; m < r; m++) {
        s1 -= pq.UU[k * R + m] * sm.X[m * r + l];
        s2 -= pq.UV[m * R + k] * sm.X[m * r + l];
      }
      sm.UCV[t] = s1;
      sm.VCV[t] = s2;
    }
    __syncthreads();
    // (VCV - delta I) c2 = V^T g - (U^T V)^T y1 ; c1 = y1 - X c2
    for (int t = threadIdx.x; t < r * r; t += blockDim.x) {
      const int k = t / r, l = t - k * r;
      sm.tmp[t] = sm.VCV[t] - (k == l ? dl : 0.0);
    }
    for (int k = threadIdx.x; k < r; k += blockDim.x) {
      double v = sm.wg[r + k];
      for (int m = 0; m < r; m++) v -= pq.UV[m * R + k] * sm.XS[m * (r + 1) + r];
      sm.c[k] = v;
    }
    __syncthreads();
    pivot_solve<double>(sm.tmp, r, sm.c, 1, r, 1, sm.cw + r, 1, sm.perm, sm.used);
    for (int k = threadIdx.x; k < r; k += blockDim.x) {
      double v = sm.XS[k * (r + 1) + r];
      for (int m = 0; m < r; m++) v -= sm.X[k * r + m] * sm.cw[r + m];
      sm.cw[k] = v;
    }
    __syncthreads();
    // x_tilde = x - (g - U c1 - V c2) / delta
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      double w = pq.g[i];
      for (int k = 0; k < r; k++) w -= pq.U[(size_t)k * n + i] * sm.cw[k] + pq.V[(size_t)k * n + i] * sm.cw[r + k];
      pq.xt[i] = pq.x[i] - idl * w;
    }
    __syncthreads();
  }
  const int it = prox_ssn(pq, wk, r, pq.xt, pq.xh, sm, red, jmax);
  double part = 0.0, amax = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double p = pq.xh[i] - pq.x[i];
    pq.p[i] = p;
    part += p * pq.g[i];
  }
  double pg = block_sum(part, red);
  int flag = 0;
  if (!(pg < 0.0)) {
    flag = 2;
    part = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const double p = fmax(pq.x[i] - pq.g[i], 0.0) - pq.x[i];
      pq.p[i] = p;
      part += p * pq.g[i];
    }
    pg = block_sum(part, red);
    __syncthreads();
    if (threadIdx.x == 0) *pq.r = 0;
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) amax = fmax(amax, fabs(pq.p[i]));
  amax = block_sum(amax > 0.0 ? 1.0 : 0.0, red);
  if (threadIdx.x == 0) {
    pq.scal[S_FLAG] = (amax == 0.0) ? 1.0 : (double)flag;
    pq.scal[S_PG] = pg;
    pq.scal[S_SSN_IT] += it < 0 ? -it : it;
    if (it < 0) pq.scal[S_SSN_FAIL] += 1.0;
  }
}

// Append (s, y) as pair number r (already checked) and its unrolled u, v.
__device__ void append_pair(PqnDev& pq, PqnWork& wk, int r, const double* s, const double* y, double ys, double sBs,
                            const double* Bs, double* red, double* tmp) {
  const int n = pq.n, R = pq.rmax;
  const double iu = 1.0 / sqrt(ys), iv = 1.0 / sqrt(sBs);
  double* Sr = pq.S + (size_t)r * n;
  double* Yr = pq.Y + (size_t)r * n;
  double* Ur = pq.U + (size_t)r * n;
  double* Vr = pq.V + (size_t)r * n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    Sr[i] = s[i];
    Yr[i] = y[i];
    Ur[i] = y[i] * iu;
    Vr[i] = Bs[i] * iv;
    wk.U32[(size_t)r * n + i] = (float)Ur[i];
    wk.V32[(size_t)r * n + i] = (float)Vr[i];
  }
  __syncthreads();
  if (threadIdx.x == 0) wk.ys[r] = ys;
  // Grams: new row/column r of UU, UV, VV
  bmultidot(pq.U, n, r + 1, Ur, tmp);            // U_k . u
  bmultidot(pq.V, n, r + 1, Ur, tmp + 64);       // V_k . u
  bmultidot(pq.U, n, r + 1, Vr, tmp + 128);      // U_k . v
  bmultidot(pq.V, n, r + 1, Vr, tmp + 192);      // V_k . v
  for (int k = threadIdx.x; k <= r; k += blockDim.x) {
    pq.UU[k * R + r] = tmp[k];
    pq.UU[r * R + k] = tmp[k];
    pq.UV[k * R + r] = tmp[128 + k];   // U_k . v_r
    pq.UV[r * R + k] = tmp[64 + k];    // u_r . V_k
    pq.VV[k * R + r] = tmp[192 + k];
    pq.VV[r * R + k] = tmp[192 + k];
  }
  __syncthreads();
}

// Bs = s + U (U^T s) - V (V^T s) for the first r pairs; returns s^T Bs.
__device__ double apply_B(const PqnDev& pq, int r, const double* s, double* Bs, double* tmp, double* red) {
  const int n = pq.n;
  bmultidot(pq.U, n, r, s, tmp);
  bmultidot(pq.V, n, r, s, tmp + 64);
  double part = 0.0;
  const double dl = delta_of(pq);
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double v = dl * s[i];
    for (int k = 0; k < r; k++) v += pq.U[(size_t)k * n + i] * tmp[k] - pq.V[(size_t)k * n + i] * tmp[64 + k];
    Bs[i] = v;
    part += s[i] * v;
  }
  return block_sum(part, red);
}

// Rebuild U, V, the Grams and y^T s from the r stored pairs (in order),
// dropping pairs that fail the curvature test.  Returns the pairs kept.
__device__ int rebuild(PqnDev& pq, PqnWork& wk, int r, double* red, double* tmp) {
  const int n = pq.n;
  int kept = 0;
  for (int k = 0; k < r; k++) {
    const double* s = pq.S + (size_t)k * n;
    const double* y = pq.Y + (size_t)k * n;
    double p1 = 0.0, p2 = 0.0, p3 = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) { p1 += y[i] * s[i]; p2 += s[i] * s[i]; p3 += y[i] * y[i]; }
    const double ys = block_sum(p1, red), ss = block_sum(p2, red), yy = block_sum(p3, red);
    const double sBs = apply_B(pq, kept, s, wk.q, tmp, red);
    if (ys > 1e-12 * sqrt(ss) * sqrt(yy) && sBs > 0.0) {
      // copy pair k to slot kept (k >= kept) before appending
      if (kept != k) {
        for (int i = threadIdx.x; i < n; i += blockDim.x) { wk.d[i] = s[i]; wk.z[i] = y[i]; }
        __syncthreads();
        append_pair(pq, wk, kept, wk.d, wk.z, ys, sBs, wk.q, red, tmp);
      } else {
        for (int i = threadIdx.x; i < n; i += blockDim.x) { wk.d[i] = s[i]; wk.z[i] = y[i]; }
        __syncthreads();
        append_pair(pq, wk, kept, wk.d, wk.z, ys, sBs, wk.q, red, tmp);
      }
      kept++;
    }
  }
  return kept;
}

__global__ void __launch_bounds__(PQN_T) k_pqn_rebuild(PqnDev pq, PqnWork wk) {
  __shared__ double red[32];
  __shared__ double tmp[256];
  const int r = *pq.r;
  __syncthreads();
  const int kept = rebuild(pq, wk, r, red, tmp);
  if (threadIdx.x == 0) *pq.r = kept;
}

// Step of Algorithm 1 after the MVP Ap = A[p] (and lop = A_hat[p] when the
// extra accumulation of Appendix D.2 is tracked): Algorithm 2, the updates of
// x and g, and the BFGS update.  quasi_newton = 0 skips the BFGS update.
__global__ void __launch_bounds__(PQN_T) k_pqn_step(PqnDev pq, PqnWork wk, int track_extra, int quasi_newton,
                                                    int scale0) {
  __shared__ double red[32];
  __shared__ double tmp[256];
  __shared__ double bestv[PQN_W];
  __shared__ int besti[PQN_W];
  const int n = pq.n;
  // Algorithm 2
  double p1 = 0.0, p2 = 0.0;
  double ev = INFINITY;
  int ei = 0x7fffffff;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double p = pq.p[i];
    p1 += p * pq.g[i];
    p2 += p * pq.Ap[i];
    if (p < 0.0) {
      const double e = -pq.x[i] / p;
      if (e < ev || (e == ev && i < ei)) { ev = e; ei = i; }
    }
  }
  const double pg = block_sum(p1, red), pAp = block_sum(p2, red);
  // (value, index) minimum
  for (int o = 16; o > 0; o >>= 1) {
    const double ov = __shfl_xor_sync(0xffffffffu, ev, o);
    const int oi = __shfl_xor_sync(0xffffffffu, ei, o);
    if (ov < ev || (ov == ev && oi < ei)) { ev = ov; ei = oi; }
  }
  if ((threadIdx.x & 31) == 0) { bestv[threadIdx.x >> 5] = ev; besti[threadIdx.x >> 5] = ei; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = bestv[0];
    int id = besti[0];
    for (int w = 1; w < PQN_W; w++)
      if (bestv[w] < v || (bestv[w] == v && besti[w] < id)) { v = bestv[w]; id = besti[w]; }
    double eta = -pg / pAp;
    int blk = -1;
    if (v < eta) { eta = v; blk = id; }
    red[0] = eta;
    red[1] = (double)blk;
    pq.scal[S_ETA] = eta;
    pq.scal[S_PAP] = pAp;
    pq.scal[S_BLK] = blk;
  }
  __syncthreads();
  const double eta = red[0];
  const int blk = (int)red[1];
  __syncthreads();
  // x, g updates; s = eta p (in wk.d), y = eta Ap (in wk.z)
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double xn = fmax(pq.x[i] + eta * pq.p[i], 0.0);
    if (i == blk) xn = 0.0;
    pq.x[i] = xn;
    pq.g[i] += eta * pq.Ap[i];
    if (track_extra) pq.extra[i] += eta * pq.lop[i];
    wk.d[i] = eta * pq.p[i];
    wk.z[i] = eta * pq.Ap[i];
  }
  __syncthreads();
  double accepted = 0.0;
  if (quasi_newton) {
    int r = *pq.r;
    double a1 = 0.0, a2 = 0.0, a3 = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      a1 += wk.z[i] * wk.d[i];
      a2 += wk.d[i] * wk.d[i];
      a3 += wk.z[i] * wk.z[i];
    }
    const double ys = block_sum(a1, red), ss = block_sum(a2, red), yy = block_sum(a3, red);
    if (scale0 && r == 0 && pq.scal[S_DSET] == 0.0 && ys > 0.0 && ss > 0.0) {
      // B_0 = delta I with delta = y^T s / s^T s of the first step
      __syncthreads();
      if (threadIdx.x == 0) {
        pq.scal[S_DELTA] = ys / ss;
        pq.scal[S_DSET] = 1.0;
      }
      __syncthreads();
    }
    const double sBs = apply_B(pq, r, wk.d, wk.q, tmp, red);
    if (ys > 1e-12 * sqrt(ss) * sqrt(yy) && sBs > 0.0) {
      accepted = 1.0;
      if (r < pq.rmax) {
        append_pair(pq, wk, r, wk.d, wk.z, ys, sBs, wk.q, red, tmp);
        r++;
      } else {
        // memory full: drop the oldest quarter of the pairs at once (so the
        // unrolled factors are rebuilt once per rmax/4 steps), append, rebuild
        const int drop = max(1, pq.rmax / 4);
        for (int k = 0; k + drop < r; k++) {
          for (int i = threadIdx.x; i < n; i += blockDim.x) {
            pq.S[(size_t)k * n + i] = pq.S[(size_t)(k + drop) * n + i];
            pq.Y[(size_t)k * n + i] = pq.Y[(size_t)(k + drop) * n + i];
          }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
          pq.S[(size_t)(r - drop) * n + i] = wk.d[i];
          pq.Y[(size_t)(r - drop) * n + i] = wk.z[i];
        }
        __syncthreads();
        r = rebuild(pq, wk, r - drop + 1, red, tmp);
      }
      __syncthreads();
      if (threadIdx.x == 0) *pq.r = r;
    }
  }
  // KKT of the new iterate
  p1 = 0.0;
  p2 = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double m = fmin(pq.x[i], pq.g[i]);
    p1 += m * m;
    p2 += pq.x[i] * pq.g[i];
  }
  const double k1 = block_sum(p1, red), k2 = block_sum(p2, red);
  if (threadIdx.x == 0) {
    pq.scal[S_KKT] = sqrt(k1);
    pq.scal[S_KKTDOT] = k2;
    pq.scal[S_ACCEPT] = accepted;
  }
}

// Bi-PQN subproblem MVP: out = lo + U_h (U_h^T v) - V_h (V_h^T v) (B^(k) of Eq. bifi-qnapprox).
__global__ void __launch_bounds__(PQN_T) k_bi_lowrank(int n, int nh, const double* Uh, const double* Vh,
                                                      const double* v, const double* lo, double* out) {
  __shared__ double c[256];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int k = w; k < 2 * nh; k += PQN_W) {
    const double* m = (k < nh ? Uh : Vh) + (size_t)(k % nh) * n;
    double s = 0.0;
    for (int i = lane; i < n; i += 32) s += m[i] * v[i];
    s = warp_sum(s);
    if (lane == 0) c[k] = s;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double s = lo[i];
    for (int k = 0; k < nh; k++) s += Uh[(size_t)k * n + i] * c[k] - Vh[(size_t)k * n + i] * c[nh + k];
    out[i] = s;
  }
}

// Bi-PQN outer update (Algorithm 4 after the high-fidelity MVP A[p]):
// Algorithm 2, x and g updates, the high-fidelity BFGS correction with
// B^(k) s = eta * ahs + U_h U_h^T s - V_h V_h^T s, and the secant carry-over
// of the subproblem pairs: Y <- Y + u (u^T S) - v (v^T S).
__global__ void __launch_bounds__(PQN_T) k_bi_outer(PqnDev out, PqnDev in, PqnWork wk, double* Uh, double* Vh,
                                                    int* nh_dev, int nh_max, const double* ahs) {
  __shared__ double red[32];
  __shared__ double c[256];
  __shared__ double bestv[PQN_W];
  __shared__ int besti[PQN_W];
  const int n = out.n;
  double p1 = 0.0, p2 = 0.0, ev = INFINITY;
  int ei = 0x7fffffff;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double p = out.p[i];
    p1 += p * out.g[i];
    p2 += p * out.Ap[i];
    if (p < 0.0) {
      const double e = -out.x[i] / p;
      if (e < ev || (e == ev && i < ei)) { ev = e; ei = i; }
    }
  }
  const double pg = block_sum(p1, red), pAp = block_sum(p2, red);
  for (int o = 16; o > 0; o >>= 1) {
    const double ov = __shfl_xor_sync(0xffffffffu, ev, o);
    const int oi = __shfl_xor_sync(0xffffffffu, ei, o);
    if (ov < ev || (ov == ev && oi < ei)) { ev = ov; ei = oi; }
  }
  if ((threadIdx.x & 31) == 0) { bestv[threadIdx.x >> 5] = ev; besti[threadIdx.x >> 5] = ei; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = bestv[0];
    int id = besti[0];
    for (int w = 1; w < PQN_W; w++)
      if (bestv[w] < v || (bestv[w] == v && besti[w] < id)) { v = bestv[w]; id = besti[w]; }
    double eta = -pg / pAp;
    int blk = -1;
    if (v < eta) { eta = v; blk = id; }
    red[0] = eta;
    red[1] = (double)blk;
    out.scal[S_ETA] = eta;
    out.scal[S_BLK] = blk;
  }
  __syncthreads();
  const double eta = red[0];
  const int blk = (int)red[1];
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double xn = fmax(out.x[i] + eta * out.p[i], 0.0);
    if (i == blk) xn = 0.0;
    out.x[i] = xn;
    out.g[i] += eta * out.Ap[i];
    wk.d[i] = eta * out.p[i];     // s
    wk.z[i] = eta * out.Ap[i];    // y
  }
  __syncthreads();
  const int nh = *nh_dev;
  // Bs = eta * ahs + U_h U_h^T s - V_h V_h^T s
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int k = w; k < 2 * nh; k += PQN_W) {
    const double* m = (k < nh ? Uh : Vh) + (size_t)(k % nh) * n;
    double s = 0.0;
    for (int i = lane; i < n; i += 32) s += m[i] * wk.d[i];
    s = warp_sum(s);
    if (lane == 0) c[k] = s;
  }
  __syncthreads();
  double a1 = 0.0, a2 = 0.0, a3 = 0.0, a4 = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double v = eta * ahs[i];
    for (int k = 0; k < nh; k++) v += Uh[(size_t)k * n + i] * c[k] - Vh[(size_t)k * n + i] * c[nh + k];
    wk.q[i] = v;
    a1 += wk.z[i] * wk.d[i];
    a2 += wk.d[i] * v;
    a3 += wk.d[i] * wk.d[i];
    a4 += wk.z[i] * wk.z[i];
  }
  const double ys = block_sum(a1, red), sBs = block_sum(a2, red), ss = block_sum(a3, red), yy = block_sum(a4, red);
  int accepted = 0;
  if (ys > 1e-12 * sqrt(ss) * sqrt(yy) && sBs > 0.0 && nh < nh_max) {
    accepted = 1;
    const double iu = 1.0 / sqrt(ys), iv = 1.0 / sqrt(sBs);
    double* u = Uh + (size_t)nh * n;
    double* v = Vh + (size_t)nh * n;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      u[i] = wk.z[i] * iu;
      v[i] = wk.q[i] * iv;
    }
    __syncthreads();
    // carry-over of the subproblem pairs held in `in`
    const int r = *in.r;
    bmultidot(in.S, n, r, u, c);         // u^T S_k
    bmultidot(in.S, n, r, v, c + 128);   // v^T S_k
    for (int k = 0; k < r; k++)
      for (int i = threadIdx.x; i < n; i += blockDim.x)
        in.Y[(size_t)k * n + i] += u[i] * c[k] - v[i] * c[128 + k];
    __syncthreads();
    if (threadIdx.x == 0) *nh_dev = nh + 1;
  }
  p1 = 0.0;
  p2 = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double m = fmin(out.x[i], out.g[i]);
    p1 += m * m;
    p2 += out.x[i] * out.g[i];
  }
  const double k1 = block_sum(p1, red), k2 = block_sum(p2, red);
  if (threadIdx.x == 0) {
    out.scal[S_KKT] = sqrt(k1);
    out.scal[S_KKTDOT] = k2;
    out.scal[S_ACCEPT] = accepted;
  }
}

// p = x_sub - x (subproblem result minus the outer iterate); p^T g; falls back
// to the projected-gradient direction when p is not a descent direction.
__global__ void __launch_bounds__(PQN_T) k_bi_direction(PqnDev out, const double* xsub) {
  __shared__ double red[32];
  const int n = out.n;
  double part = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double p = xsub[i] - out.x[i];
    out.p[i] = p;
    part += p * out.g[i];
  }
  double pg = block_sum(part, red);
  double flag = 0.0;
  if (!(pg < 0.0)) {
    flag = 2.0;
    part = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const double p = fmax(out.x[i] - out.g[i], 0.0) - out.x[i];
      out.p[i] = p;
      part += p * out.g[i];
    }
    pg = block_sum(part, red);
  }
  double nz = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) nz += out.p[i] != 0.0 ? 1.0 : 0.0;
  nz = block_sum(nz, red);
  if (threadIdx.x == 0) {
    out.scal[S_FLAG] = nz == 0.0 ? 1.0 : flag;
    out.scal[S_PG] = pg;
  }
}

// M D x accumulated with the same over-relaxation as the gradient (the MVP
// reuse of Sec. 4 applied to the 6M body velocities): init copies, else adds
// eta * (M D p) with eta read from the PQN scalars.
__global__ void k_mdx(int m6, const double* __restrict__ uo, const double* __restrict__ scal, int init,
                      double* __restrict__ mdx) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m6) return;
  mdx[i] = init ? uo[i] : mdx[i] + scal[S_ETA] * uo[i];
}

// BB-PGD (Sec. 6, Eq. spectralStepSize; Table 1: over-relaxation 1):
// p = (x - tau g)_+ - x.
__global__ void __launch_bounds__(PQN_T) k_pgd_direction(PqnDev pq) {
  __shared__ double red[32];
  const double tau = pq.scal[S_TAU];
  double nz = 0.0;
  for (int i = threadIdx.x; i < pq.n; i += blockDim.x) {
    const double p = fmax(pq.x[i] - tau * pq.g[i], 0.0) - pq.x[i];
    pq.p[i] = p;
    nz += p != 0.0 ? 1.0 : 0.0;
  }
  nz = block_sum(nz, red);
  if (threadIdx.x == 0) pq.scal[S_FLAG] = nz == 0.0 ? 1.0 : 0.0;
}

// x += p, g += A p, tau = p^T p / p^T A p (tau0 if not positive), KKT.
__global__ void __launch_bounds__(PQN_T) k_pgd_step(PqnDev pq, double tau0) {
  __shared__ double red[32];
  double a = 0.0, c = 0.0, k1 = 0.0, k2 = 0.0;
  for (int i = threadIdx.x; i < pq.n; i += blockDim.x) {
    const double p = pq.p[i], ap = pq.Ap[i];
    a += p * p;
    c += p * ap;
    const double x = fmax(pq.x[i] + p, 0.0);
    const double g = pq.g[i] + ap;
    pq.x[i] = x;
    pq.g[i] = g;
    const double m = fmin(x, g);
    k1 += m * m;
    k2 += x * g;
  }
  a = block_sum(a, red);
  c = block_sum(c, red);
  k1 = block_sum(k1, red);
  k2 = block_sum(k2, red);
  if (threadIdx.x == 0) {
    pq.scal[S_TAU] = c > 0.0 ? a / c : tau0;
    pq.scal[S_ETA] = 1.0;
    pq.scal[S_KKT] = sqrt(k1);
    pq.scal[S_KKTDOT] = k2;
  }
}

__global__ void k_set_scalar(double* slot, double v) { *slot = v; }

__global__ void k_copy(int n, const double* a, double* b) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = a[i];
}
__global__ void k_zero(int n, double* a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] = 0.0;
}

// ------------------------------------------------------------------ host side
struct PqnHost {
  PqnDev d;
  PqnWork w;
};

static PqnWork work_of(lcp_ctx* ctx, const PqnDev& pq);

static size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }

// Bytes of the device state of one PQN run with n contacts and rmax pairs.
size_t pqn_bytes(int n, int rmax) {
  const size_t nn = n > 0 ? n : 1;
  return 8 * al256(sizeof(double) * nn) + 4 * al256(sizeof(double) * nn * rmax) +
         3 * al256(sizeof(double) * rmax * rmax) + al256(sizeof(int) * 4) +
         al256(sizeof(double) * (S_NSCAL + 4 * nn + 2 * nn * rmax + rmax));
}

// Lays the state out from base; returns the first byte after it.
char* pqn_carve(PqnDev* pq, char* base, int n, int rmax) {
  const size_t nn = n > 0 ? n : 1;
  pq->n = n;
  pq->rmax = rmax;
  double** vecs[] = {&pq->x, &pq->g, &pq->p, &pq->Ap, &pq->xt, &pq->xh, &pq->extra, &pq->lop};
  for (double** v : vecs) { *v = (double*)base; base += al256(sizeof(double) * nn); }
  double** mats[] = {&pq->S, &pq->Y, &pq->U, &pq->V};
  for (double** m : mats) { *m = (double*)base; base += al256(sizeof(double) * nn * rmax); }
  double** grams[] = {&pq->UU, &pq->UV, &pq->VV};
  for (double** g : grams) { *g = (double*)base; base += al256(sizeof(double) * rmax * rmax); }
  pq->r = (int*)base;
  base += al256(sizeof(int) * 4);
  pq->scal = (double*)base;
  base += al256(sizeof(double) * (S_NSCAL + 4 * nn + 2 * nn * rmax + rmax));
  return base;
}

int pqn_reset(lcp_ctx* ctx, PqnDev* pq) {
  LCP_CUDA(cudaMemsetAsync(pq->r, 0, sizeof(int) * 4, ctx->stream));
  LCP_CUDA(cudaMemsetAsync(pq->scal, 0, sizeof(double) * S_NSCAL, ctx->stream));
  return LCP_OK;
}

static PqnWork work_of(lcp_ctx* ctx, const PqnDev& pq) {
  (void)ctx;
  const int nn = pq.n > 0 ? pq.n : 1;
  PqnWork w;
  double* base = pq.scal + S_NSCAL;
  w.y = base;
  w.z = w.y + nn;
  w.d = w.z + nn;
  w.q = w.d + nn;
  float* f = (float*)(w.q + nn);
  w.U32 = f;
  w.V32 = w.U32 + (size_t)nn * pq.rmax;
  w.lam = w.V32 + (size_t)nn * pq.rmax;   // uses the slack of the 2 n rmax doubles
  w.ys = (double*)(f + 2 * (size_t)nn * pq.rmax + 2 * (size_t)nn);
  return w;
}

// host helpers -------------------------------------------------------------
static int read_scal(lcp_ctx* ctx, const PqnDev& pq, double* out) {
  LCP_CUDA(cudaMemcpyAsync(ctx->hscal + 16, pq.scal, sizeof(double) * S_NSCAL, cudaMemcpyDeviceToHost, ctx->stream));
  LCP_CUDA(cudaStreamSynchronize(ctx->stream));
  for (int k = 0; k < S_NSCAL; k++) out[k] = ctx->hscal[16 + k];
  return LCP_OK;
}

typedef int (*MvpFn)(lcp_ctx*, const double*, double*);

struct Timer {
  cudaEvent_t a, b;
};

static double now_s() {
  timespec t;
  clock_gettime(CLOCK_MONOTONIC, &t);
  return t.tv_sec + 1e-9 * t.tv_nsec;
}

// Inner MVP of Bi-PQN subproblems: lop = A_hat[v]; Ap = lop + U_h U_h^T v - V_h V_h^T v.
static int mvp_sub(lcp_ctx* ctx, PqnDev& pq, const double* v) {
  cudaEvent_t ev = prof_begin(ctx);
  LCP_TRY(mvp_low(ctx, v, pq.lop));
  prof_end(ctx, ev, 6);
  ++ctx->nlaunch, k_bi_lowrank<<<1, PQN_T, 0, ctx->stream>>>(pq.n, ctx->nh, ctx->Uh, ctx->Vh, v, pq.lop, pq.Ap);
  LCP_CUDA(cudaGetLastError());
  return LCP_OK;
}

struct RunStats {
  int iterations = 0, mvps = 0, resets = 0;
  double kkt = 0.0, kktdot = 0.0, t_mvp = 0.0;
  bool converged = false;
};

// Algorithm 1 on state pq.  mode 0: MVP = A (fidelity hi/lo via mvp), g from
// A x + b; mode 1: Bi-PQN subproblem (MVP = B^(k), g0 given, extra tracked).
// Algorithm 1 on pq; stops at ||min(x, g)|| <= max(tol, tol_rel * initial value).
static int run_mono(lcp_ctx* ctx, PqnDev& pq, MvpFn mvp, int sub, const double* b, const double* g0, double tol,
                    int kmax, RunStats* rs, double tol_rel = 0.0) {
  const bool track = !sub && mvp == mvp_high;   // body velocities M D x for the time step
  const int m6 = 6 * ctx->M;
  PqnWork wk = work_of(ctx, pq);
  double sc[S_NSCAL];
  const size_t smem = prox_smem_bytes(pq.rmax);
  double t0;
  if (!sub) {
    t0 = now_s();
    LCP_TRY(mvp(ctx, pq.x, pq.Ap));
    if (track) ++ctx->nlaunch, k_mdx<<<(m6 + 127) / 128, 128, 0, ctx->stream>>>(m6, ctx->UO, pq.scal, 1, ctx->MDx);
    LCP_CUDA(cudaStreamSynchronize(ctx->stream));
    rs->t_mvp += now_s() - t0;
    rs->mvps++;
    ++ctx->nlaunch, k_pqn_grad<<<1, PQN_T, 0, ctx->stream>>>(pq, pq.Ap, b, nullptr);
  } else {
    ++ctx->nlaunch, k_pqn_grad<<<1, PQN_T, 0, ctx->stream>>>(pq, nullptr, nullptr, g0);
  }
  LCP_CUDA(cudaGetLastError());
  LCP_TRY(read_scal(ctx, pq, sc));
  tol = std::max(tol, tol_rel * sc[S_KKT]);
  int k = 0;
  for (; k < kmax; k++) {
    if (!(sc[S_KKT] == sc[S_KKT])) { ctx->err = "PQN: NaN in the KKT error"; return LCP_ERR_NUMERICAL; }
    if (sc[S_KKT] <= tol) break;
    cudaEvent_t ev = prof_begin(ctx);
    ++ctx->nlaunch, k_pqn_direction<<<1, PQN_T, smem, ctx->stream>>>(pq, wk, ctx->cfg.ssn_maxit);
    prof_end(ctx, ev, 3);
    LCP_CUDA(cudaGetLastError());
    LCP_TRY(read_scal(ctx, pq, sc));
    if (sc[S_FLAG] == 1.0) break;  // p = 0: stationary
    if (sc[S_FLAG] == 2.0) rs->resets++;
    t0 = now_s();
    if (sub) {
      LCP_TRY(mvp_sub(ctx, pq, pq.p));
    } else {
      LCP_TRY(mvp(ctx, pq.p, pq.Ap));
    }
    LCP_CUDA(cudaStreamSynchronize(ctx->stream));
    rs->t_mvp += now_s() - t0;
    rs->mvps++;
    ev = prof_begin(ctx);
    ++ctx->nlaunch, k_pqn_step<<<1, PQN_T, 0, ctx->stream>>>(pq, wk, sub, 1, ctx->cfg.h0_scaling);
    prof_end(ctx, ev, 4);
    if (track) ++ctx->nlaunch, k_mdx<<<(m6 + 127) / 128, 128, 0, ctx->stream>>>(m6, ctx->UO, pq.scal, 0, ctx->MDx);
    LCP_CUDA(cudaGetLastError());
    LCP_TRY(read_scal(ctx, pq, sc));
  }
  rs->iterations = k;
  rs->kkt = sc[S_KKT];
  rs->kktdot = sc[S_KKTDOT];
  rs->converged = sc[S_KKT] <= tol;
  return LCP_OK;
}

int pqn_configure(lcp_ctx* ctx, int rmax) {
  const size_t smem = prox_smem_bytes(rmax);
  if (smem > 48 * 1024)
    LCP_CUDA(raise_smem_limit((const void*)k_pqn_direction, smem));
  return LCP_OK;
}

int lcp_solve_device(lcp_ctx* ctx, int method, double tol, const double* x0, double* x, lcp_stats* st) {
  const int n = ctx->n;
  const double t_start = now_s();
  ctx->c_gmres = ctx->c_fp32 = ctx->c_fp64 = ctx->c_df64 = 0;
  ctx->c_recycled = 0;
  if (ctx->lo) ctx->lo->c_gmres = ctx->lo->c_recycled = 0;
  recycle_reset(ctx);   // each LCP solve depends only on its configuration
  lcp_stats s{};
  // along a trajectory (lcp_step, cfg.warm_start & LCP_WARM_FORCES) start from the previous step's
  // forces on the contacts that persist, unless the caller gives x0
  if (!x0 && ctx->x_warm_valid) {
    x0 = ctx->x_warm;
    s.warm_x0 = 1;
  }
  ctx->x_warm_valid = false;
  s.unc_gmres_iterations = ctx->unc_its;
  s.unc_warm_started = ctx->unc_warm;
  if (n == 0) {
    LCP_CUDA(cudaMemsetAsync(ctx->MDx, 0, sizeof(double) * 6 * ctx->M, ctx->stream));
    ctx->have_solution = true;
    s.converged = 1;
    if (st) *st = s;
    return LCP_OK;
  }
  ctx->have_solution = false;
  PqnDev& po = ctx->pq_outer;
  PqnDev& pi = ctx->pq_inner;
  const int T = 256;
  int status = LCP_OK;
  LCP_CUDA(cudaMemsetAsync(po.r, 0, sizeof(int), ctx->stream));
  LCP_CUDA(cudaMemsetAsync(pi.r, 0, sizeof(int), ctx->stream));
  LCP_CUDA(cudaMemsetAsync(po.scal, 0, sizeof(double) * S_NSCAL, ctx->stream));
  LCP_CUDA(cudaMemsetAsync(pi.scal, 0, sizeof(double) * S_NSCAL, ctx->stream));
  double sc[S_NSCAL];
  if (method == LCP_MONO_PQN) {
    RunStats rs;
    ++ctx->nlaunch, k_pqn_init<<<1, PQN_T, 0, ctx->stream>>>(po, x0);
    LCP_TRY(run_mono(ctx, po, mvp_high, 0, ctx->b, nullptr, tol, ctx->cfg.kmax, &rs));
    s.iterations = rs.iterations;
    s.resets = rs.resets;
    s.hi_mvps = rs.mvps;
    s.kkt_abs = rs.kkt;
    s.kkt_dot = rs.kktdot;
    s.converged = rs.converged;
    s.hi_mvp_seconds = rs.mvps ? rs.t_mvp / rs.mvps : 0.0;
    s.e_mvps = s.hi_mvps;
    ++ctx->nlaunch, k_copy<<<(n + T - 1) / T, T, 0, ctx->stream>>>(n, po.x, x);
  } else if (method == LCP_BI_PQN) {
    // low-fidelity initialisation: Mono-PQN on A_hat from x0, its pairs kept in pi
    RunStats r0;
    ++ctx->nlaunch, k_pqn_init<<<1, PQN_T, 0, ctx->stream>>>(pi, x0);
    // LCP_WARM_NO_INIT: a start carried from the previous step is taken as x(0) as it is
    const int kinit = (s.warm_x0 && (ctx->cfg.warm_start & LCP_WARM_NO_INIT)) ? 0 : ctx->cfg.kmax_inner;
    LCP_TRY(run_mono(ctx, pi, mvp_low, 0, ctx->b, nullptr, tol, kinit, &r0, ctx->cfg.init_forcing));
    int lo = r0.mvps, hi = 0, inner_total = r0.iterations;
    s.resets = r0.resets;
    double t_lo = r0.t_mvp, t_hi = 0.0;
    ctx->nh = 0;
    int* nh_dev = (int*)(ctx->dscal + 62);
    LCP_CUDA(cudaMemsetAsync(nh_dev, 0, sizeof(int), ctx->stream));
    ++ctx->nlaunch, k_copy<<<(n + T - 1) / T, T, 0, ctx->stream>>>(n, pi.x, po.x);
    double t0 = now_s();
    LCP_TRY(mvp_high(ctx, po.x, po.Ap));
    ++ctx->nlaunch, k_mdx<<<(6 * ctx->M + 127) / 128, 128, 0, ctx->stream>>>(6 * ctx->M, ctx->UO, po.scal, 1, ctx->MDx);
    LCP_CUDA(cudaStreamSynchronize(ctx->stream));
    t_hi += now_s() - t0;
    hi++;
    ++ctx->nlaunch, k_pqn_grad<<<1, PQN_T, 0, ctx->stream>>>(po, po.Ap, ctx->b, nullptr);
    LCP_TRY(read_scal(ctx, po, sc));
    PqnWork wk_in = work_of(ctx, pi);
    int k = 0;
    for (; k < ctx->cfg.kmax; k++) {
      if (!(sc[S_KKT] == sc[S_KKT])) { ctx->err = "Bi-PQN: NaN in the KKT error"; return LCP_ERR_NUMERICAL; }
      if (sc[S_KKT] <= tol) break;
      // subproblem (Eq. pqnSubproblem) from x with gradient g, inherited pairs
      ++ctx->nlaunch, k_copy<<<(n + T - 1) / T, T, 0, ctx->stream>>>(n, po.x, pi.x);
      ++ctx->nlaunch, k_zero<<<(n + T - 1) / T, T, 0, ctx->stream>>>(n, pi.extra);
      cudaEvent_t evr = prof_begin(ctx);
      ++ctx->nlaunch, k_pqn_rebuild<<<1, PQN_T, 0, ctx->stream>>>(pi, wk_in);
      prof_end(ctx, evr, 5);
      LCP_CUDA(cudaGetLastError());
      RunStats rs;
      const double tin = std::max(0.1 * tol, ctx->cfg.forcing * sc[S_KKT]);
      LCP_TRY(run_mono(ctx, pi, nullptr, 1, nullptr, po.g, tin, ctx->cfg.kmax_inner, &rs));
      lo += rs.mvps;
      t_lo += rs.t_mvp;
      s.resets += rs.resets;
      inner_total += rs.iterations;
      ++ctx->nlaunch, k_bi_direction<<<1, PQN_T, 0, ctx->stream>>>(po, pi.x);
      LCP_TRY(read_scal(ctx, po, sc));
      if (sc[S_FLAG] == 1.0) break;
      const double* ahs = pi.extra;
      if (sc[S_FLAG] == 2.0) {   // fallback direction: A_hat p by one more low-fidelity MVP
        t0 = now_s();
        LCP_TRY(mvp_low(ctx, po.p, pi.lop));
        LCP_CUDA(cudaStreamSynchronize(ctx->stream));
        t_lo += now_s() - t0;
        lo++;
        ahs = pi.lop;
      }
      t0 = now_s();
      LCP_TRY(mvp_high(ctx, po.p, po.Ap));
      LCP_CUDA(cudaStreamSynchronize(ctx->stream));
      t_hi += now_s() - t0;
      hi++;
      ++ctx->nlaunch, k_bi_outer<<<1, PQN_T, 0, ctx->stream>>>(po, pi, wk_in, ctx->Uh, ctx->Vh, nh_dev, ctx->cfg.kmax, ahs);
      ++ctx->nlaunch, k_mdx<<<(6 * ctx->M + 127) / 128, 128, 0, ctx->stream>>>(6 * ctx->M, ctx->UO, po.scal, 0, ctx->MDx);
      LCP_CUDA(cudaGetLastError());
      int nh_host = 0;
      LCP_CUDA(cudaMemcpyAsync(&nh_host, nh_dev, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
      LCP_TRY(read_scal(ctx, po, sc));
      ctx->nh = nh_host;
    }
    s.iterations = k;
    s.hi_mvps = hi;
    s.lo_mvps = lo;
    s.inner_iterations = inner_total;
    s.kkt_abs = sc[S_KKT];
    s.kkt_dot = sc[S_KKTDOT];
    s.converged = sc[S_KKT] <= tol;
    s.hi_mvp_seconds = hi ? t_hi / hi : 0.0;
    s.lo_mvp_seconds = lo ? t_lo / lo : 0.0;
    s.e_mvps = hi + (s.hi_mvp_seconds > 0 ? lo * s.lo_mvp_seconds / s.hi_mvp_seconds : 0.0);
    ++ctx->nlaunch, k_copy<<<(n + T - 1) / T, T, 0, ctx->stream>>>(n, po.x, x);
  } else if (method == LCP_BB_PGD) {
    // BB-PGD baseline of Sec. 6: one MVP per iteration; tau_0 = 3 pi mu a
    const double tau0 = 3.0 * LCP_PI * ctx->cfg.viscosity * ctx->cfg.radius;
    const int m6 = 6 * ctx->M;
    ++ctx->nlaunch, k_pqn_init<<<1, PQN_T, 0, ctx->stream>>>(po, x0);
    double t0 = now_s(), t_hi = 0.0;
    LCP_TRY(mvp_high(ctx, po.x, po.Ap));
    ++ctx->nlaunch, k_mdx<<<(m6 + 127) / 128, 128, 0, ctx->stream>>>(m6, ctx->UO, po.scal, 1, ctx->MDx);
    LCP_CUDA(cudaStreamSynchronize(ctx->stream));
    t_hi += now_s() - t0;
    int hi = 1;
    ++ctx->nlaunch, k_pqn_grad<<<1, PQN_T, 0, ctx->stream>>>(po, po.Ap, ctx->b, nullptr);
    ++ctx->nlaunch, k_set_scalar<<<1, 1, 0, ctx->stream>>>(po.scal + S_TAU, tau0);
    LCP_TRY(read_scal(ctx, po, sc));
    int k = 0;
    for (; k < ctx->cfg.kmax; k++) {
      if (!(sc[S_KKT] == sc[S_KKT])) { ctx->err = "BB-PGD: NaN in the KKT error"; return LCP_ERR_NUMERICAL; }
      if (sc[S_KKT] <= tol) break;
      ++ctx->nlaunch, k_pgd_direction<<<1, PQN_T, 0, ctx->stream>>>(po);
      LCP_TRY(read_scal(ctx, po, sc));
      if (sc[S_FLAG] == 1.0) break;
      t0 = now_s();
      LCP_TRY(mvp_high(ctx, po.p, po.Ap));
      LCP_CUDA(cudaStreamSynchronize(ctx->stream));
      t_hi += now_s() - t0;
      hi++;
      ++ctx->nlaunch, k_pgd_step<<<1, PQN_T, 0, ctx->stream>>>(po, tau0);
      ++ctx->nlaunch, k_mdx<<<(m6 + 127) / 128, 128, 0, ctx->stream>>>(m6, ctx->UO, po.scal, 0, ctx->MDx);
      LCP_TRY(read_scal(ctx, po, sc));
    }
    s.iterations = k;
    s.hi_mvps = hi;
    s.kkt_abs = sc[S_KKT];
    s.kkt_dot = sc[S_KKTDOT];
    s.converged = sc[S_KKT] <= tol;
    s.hi_mvp_seconds = t_hi / hi;
    s.e_mvps = hi;
    ++ctx->nlaunch, k_copy<<<(n + T - 1) / T, T, 0, ctx->stream>>>(n, po.x, x);
  } else {
    ctx->err = "unknown method";
    return LCP_ERR_INVALID_ARG;
  }
  LCP_CUDA(cudaGetLastError());
  LCP_CUDA(cudaStreamSynchronize(ctx->stream));
  {
    double a[S_NSCAL], b2[S_NSCAL];
    LCP_TRY(read_scal(ctx, po, a));
    LCP_TRY(read_scal(ctx, pi, b2));
    s.ssn_iterations = (int)(a[S_SSN_IT] + b2[S_SSN_IT]);
    s.ssn_fallbacks = (int)(a[S_SSN_FAIL] + b2[S_SSN_FAIL]);
    s.h0_delta = method == LCP_BI_PQN ? (b2[S_DSET] != 0.0 ? b2[S_DELTA] : 1.0)
                                      : (a[S_DSET] != 0.0 ? a[S_DELTA] : 1.0);
  }
  s.gmres_iterations = ctx->c_gmres;
  s.lo_gmres_iterations = ctx->lo ? ctx->lo->c_gmres : 0;
  s.recycled_solves = ctx->c_recycled + (ctx->lo ? ctx->lo->c_recycled : 0);
  s.fp32_applies = ctx->c_fp32;
  s.fp64_applies = ctx->c_fp64;
  s.df64_applies = ctx->c_df64;
  s.seconds = now_s() - t_start;
  if (st) *st = s;
  ctx->have_solution = true;
  if (!s.converged) {
    ctx->err = "PQN reached its iteration limit";
    status = LCP_ERR_NOT_CONVERGED;
  }
  return status;
}
