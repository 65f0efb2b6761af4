// High-order quadrature of each sphere's self-interaction (cfg.self_quadrature).
//
// The pair sums evaluate the double layer of a sphere on its own nodes with
// the product rule and the global singularity subtraction, (K phi)_p =
// sum_{q != p} w_q T(x_p - x_q, n_q)(phi_q - phi_p).  That is exact on rigid
// motions but only algebraically accurate for other densities.  All spheres
// carry the same template, so one dense 3 ns x 3 ns correction C = S_acc -
// S_plain serves every body: out_b += C phi_b.
//
// S_acc: for each target node p the integral over the sphere is taken on a
// polar grid whose pole is x_p (Gauss-Legendre in the polar angle on (0, pi),
// uniform in the azimuth).  On a sphere (x - y).n(y) = -|x - y|^2 / (2a), so
// the kernel is O(1/|x - y|) and the polar area element a^2 sin(theta) cancels
// it: the rule converges spectrally.  The density at the grid points is the
// band-limited projection of the nodal values (degree <= n_theta - 1), by the
// addition theorem sum_l (2l + 1)/(4 pi) P_l(cos gamma) with the template's
// quadrature weights.  S_plain is the product rule above.  Built on the host
// in FP64 once per (grid, radius) and process, kept in FP32 (for the FP32
// sums) and FP64 (for the FP64 and double-FP32 sums).
#include <algorithm>
#include <cmath>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <tuple>
#include <vector>

#include "common.cuh"

namespace {

// Gauss-Legendre nodes and weights on [-1, 1]: Newton's method on P_n from the
// usual cosine estimates of its roots.
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < n; i++) {
    double t = std::cos(LCP_PI * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; it++) {
      double p0 = 1.0, p1 = t;
      for (int k = 1; k < n; k++) {
        const double p2 = ((2 * k + 1) * t * p1 - k * p0) / (k + 1);
        p0 = p1;
        p1 = p2;
      }
      dp = n * (t * p1 - p0) / (t * t - 1.0);
      const double dt = p1 / dp;
      t -= dt;
      if (std::fabs(dt) < 1e-16) break;
    }
    double p0 = 1.0, p1 = t;
    for (int k = 1; k < n; k++) {
      const double p2 = ((2 * k + 1) * t * p1 - k * p0) / (k + 1);
      p0 = p1;
      p1 = p2;
    }
    dp = n * (t * p1 - p0) / (t * t - 1.0);
    x[i] = t;
    w[i] = 2.0 / ((1.0 - t * t) * dp * dp);
  }
}

struct Template {
  int ns = 0;
  double a = 1.0;
  std::vector<double> xi, w;   // [ns][3] node positions (relative to the centre), [ns] weights
};

// Rows 3p..3p+2 of S_acc - S_plain for targets p in [p0, p1).
void correction_rows(const Template& tp, int L, int nr, int np, int p0, int p1, std::vector<double>& C) {
  const int ns = tp.ns, n = 3 * ns;
  const double a = tp.a, c = -3.0 / (4.0 * LCP_PI);
  std::vector<double> gx, gw;
  gauss_legendre(nr, gx, gw);
  std::vector<double> xhat(3 * ns);
  for (int q = 0; q < ns; q++)
    for (int d = 0; d < 3; d++) xhat[3 * q + d] = tp.xi[3 * q + d] / a;
  std::vector<double> coefl(L + 1);
  for (int l = 0; l <= L; l++) coefl[l] = (2 * l + 1) / (4.0 * LCP_PI);
  std::vector<double> interp(ns);
  for (int p = p0; p < p1; p++) {
    double* Cp = &C[(size_t)3 * p * n];   // three rows
    const double* xp = &tp.xi[3 * p];
    const double e[3] = {xp[0] / a, xp[1] / a, xp[2] / a};
    const double h[3] = {std::fabs(e[0]) < 0.9 ? 1.0 : 0.0, std::fabs(e[0]) < 0.9 ? 0.0 : 1.0, 0.0};
    double t1[3] = {e[1] * h[2] - e[2] * h[1], e[2] * h[0] - e[0] * h[2], e[0] * h[1] - e[1] * h[0]};
    const double t1n = std::sqrt(t1[0] * t1[0] + t1[1] * t1[1] + t1[2] * t1[2]);
    for (int d = 0; d < 3; d++) t1[d] /= t1n;
    const double t2[3] = {e[1] * t1[2] - e[2] * t1[1], e[2] * t1[0] - e[0] * t1[2], e[0] * t1[1] - e[1] * t1[0]};
    double diag[9] = {0.0};
    // S_acc: the polar grid about x_p
    for (int i = 0; i < nr; i++) {
      const double th = 0.5 * LCP_PI * (gx[i] + 1.0), wth = 0.5 * LCP_PI * gw[i];
      const double st = std::sin(th), ct = std::cos(th);
      for (int k = 0; k < np; k++) {
        const double ph = 2.0 * LCP_PI * k / np;
        const double cp = std::cos(ph), sp = std::sin(ph);
        double dir[3];
        for (int d = 0; d < 3; d++) dir[d] = ct * e[d] + st * (cp * t1[d] + sp * t2[d]);
        const double W = a * a * st * wth * (2.0 * LCP_PI / np);
        const double r[3] = {xp[0] - a * dir[0], xp[1] - a * dir[1], xp[2] - a * dir[2]};
        const double r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
        const double rn = r[0] * dir[0] + r[1] * dir[1] + r[2] * dir[2];
        const double coef = c * W * rn / (r2 * r2 * std::sqrt(r2));
        double blk[9];
        for (int u = 0; u < 3; u++)
          for (int v = 0; v < 3; v++) blk[3 * u + v] = coef * r[u] * r[v];
        for (int u = 0; u < 9; u++) diag[u] += blk[u];
        // density at dir: the band-limited projection of the nodal values
        for (int q = 0; q < ns; q++) {
          const double mu = dir[0] * xhat[3 * q] + dir[1] * xhat[3 * q + 1] + dir[2] * xhat[3 * q + 2];
          double pm1 = 1.0, pl = mu, s = coefl[0] + coefl[1] * mu;
          for (int l = 2; l <= L; l++) {
            const double pn = ((2 * l - 1) * mu * pl - (l - 1) * pm1) / l;
            pm1 = pl;
            pl = pn;
            s += coefl[l] * pl;
          }
          interp[q] = (L >= 1 ? s : coefl[0]) * tp.w[q] / (a * a);
        }
        for (int q = 0; q < ns; q++) {
          const double f = interp[q];
          for (int u = 0; u < 3; u++)
            for (int v = 0; v < 3; v++) Cp[(size_t)u * n + 3 * q + v] += blk[3 * u + v] * f;
        }
      }
    }
    for (int u = 0; u < 3; u++)
      for (int v = 0; v < 3; v++) Cp[(size_t)u * n + 3 * p + v] -= diag[3 * u + v];
    // minus S_plain: the product rule with the subtraction, as the pair sums take it
    double pdiag[9] = {0.0};
    for (int q = 0; q < ns; q++) {
      if (q == p) continue;
      const double* xq = &tp.xi[3 * q];
      const double r[3] = {xp[0] - xq[0], xp[1] - xq[1], xp[2] - xq[2]};
      const double r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
      const double rn = (r[0] * xq[0] + r[1] * xq[1] + r[2] * xq[2]) / a;
      const double coef = c * tp.w[q] * rn / (r2 * r2 * std::sqrt(r2));
      for (int u = 0; u < 3; u++)
        for (int v = 0; v < 3; v++) {
          const double b = coef * r[u] * r[v];
          Cp[(size_t)u * n + 3 * q + v] -= b;
          pdiag[3 * u + v] += b;
        }
    }
    for (int u = 0; u < 3; u++)
      for (int v = 0; v < 3; v++) Cp[(size_t)u * n + 3 * p + v] += pdiag[3 * u + v];
  }
}

std::mutex g_self_mu;
std::map<std::tuple<int, int, double>, std::shared_ptr<const std::vector<double>>> g_self_cache;

// The correction of a (grid, radius), built once per process (row-major n x n).
std::shared_ptr<const std::vector<double>> correction(const Template& tp, int nt, int nph) {
  const auto key = std::make_tuple(nt, nph, tp.a);
  {
    std::lock_guard<std::mutex> lock(g_self_mu);
    auto it = g_self_cache.find(key);
    if (it != g_self_cache.end()) return it->second;
  }
  const int ns = tp.ns, n = 3 * ns, L = nt - 1;
  const int nr = 2 * nt + 2, np = 4 * nt + 4;   // polar grid about each node
  auto C = std::make_shared<std::vector<double>>((size_t)n * n, 0.0);
  const int nthreads = std::max(1, std::min<int>(16, (int)std::thread::hardware_concurrency()));
  std::vector<std::thread> pool;
  const int chunk = (ns + nthreads - 1) / nthreads;
  for (int t = 0; t < nthreads; t++) {
    const int p0 = t * chunk, p1 = std::min(ns, p0 + chunk);
    if (p0 >= p1) break;
    pool.emplace_back([&, p0, p1]() { correction_rows(tp, L, nr, np, p0, p1, *C); });
  }
  for (auto& th : pool) th.join();
  std::lock_guard<std::mutex> lock(g_self_mu);
  g_self_cache.emplace(key, C);
  return C;
}

}  // namespace

// out_b += C phi_b for every body b, FP64 (C stored transposed: Ct[j * n + i] =
// C[i][j], so that the threads of a block read consecutive entries).
__global__ void k_self64(int n, int M, const double* __restrict__ Ct, const double* __restrict__ phi,
                         double* __restrict__ out) {
  extern __shared__ double vb[];
  const int b = blockIdx.y;
  for (int j = threadIdx.x; j < n; j += blockDim.x) vb[j] = phi[(size_t)b * n + j];
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = 0.0;
  for (int j = 0; j < n; j++) s = fma(Ct[(size_t)j * n + i], vb[j], s);
  out[(size_t)b * n + i] += s;
}

// The template on the host: Gauss-Legendre in t = cos(theta) ascending, uniform
// azimuth, node q = j n_phi + k (the order of the device template).
static Template host_template(int nt, int nph, double a) {
  Template tp;
  tp.ns = nt * nph;
  tp.a = a;
  std::vector<double> gx, gw;
  gauss_legendre(nt, gx, gw);   // descending roots
  tp.xi.resize(3 * (size_t)tp.ns);
  tp.w.resize(tp.ns);
  for (int j = 0; j < nt; j++) {
    const double t = gx[nt - 1 - j], wt = gw[nt - 1 - j], st = std::sqrt(1.0 - t * t);
    for (int k = 0; k < nph; k++) {
      const double ph = 2.0 * LCP_PI * k / nph;
      const int q = j * nph + k;
      tp.xi[3 * q] = a * st * std::cos(ph);
      tp.xi[3 * q + 1] = a * st * std::sin(ph);
      tp.xi[3 * q + 2] = a * t;
      tp.w[q] = a * a * wt * 2.0 * LCP_PI / nph;
    }
  }
  return tp;
}

extern "C" int lcp_self_correction(int n_theta, int n_phi, double radius, double* C) {
  if (n_theta < 2 || n_phi < 4 || (n_phi & 1) || n_theta * n_phi > 512 || !(radius > 0) || !C)
    return LCP_ERR_INVALID_ARG;
  const Template tp = host_template(n_theta, n_phi, radius);
  const auto M = correction(tp, n_theta, n_phi);
  std::copy(M->begin(), M->end(), C);
  return LCP_OK;
}

int self_correction_build(lcp_ctx* ctx) {
  const int ns = ctx->ns, n = 3 * ns;
  Template tp;
  tp.ns = ns;
  tp.a = ctx->cfg.radius;
  std::vector<double> h((size_t)8 * ns);
  LCP_CUDA(cudaMemcpyAsync(h.data(), ctx->tmpl64, sizeof(double) * 8 * ns, cudaMemcpyDeviceToHost, ctx->stream));
  LCP_CUDA(cudaStreamSynchronize(ctx->stream));
  tp.xi.resize(3 * (size_t)ns);
  tp.w.resize(ns);
  for (int q = 0; q < ns; q++) {
    for (int d = 0; d < 3; d++) tp.xi[3 * q + d] = h[8 * q + d];
    tp.w[q] = h[8 * q + 6];
  }
  const auto C = correction(tp, ctx->cfg.n_theta, ctx->cfg.n_phi);
  std::vector<float> c32((size_t)n * n);
  std::vector<double> ct((size_t)n * n);
  for (int i = 0; i < n; i++)
    for (int j = 0; j < n; j++) {
      const double v = (*C)[(size_t)i * n + j];
      c32[(size_t)i * n + j] = (float)v;
      ct[(size_t)j * n + i] = v;
    }
  ctx->cself32 = (float*)ctx_alloc(ctx, sizeof(float) * (size_t)n * n);
  ctx->cself64t = (double*)ctx_alloc(ctx, sizeof(double) * (size_t)n * n);
  if (!ctx->cself32 || !ctx->cself64t) return LCP_ERR_OOM;
  LCP_CUDA(cudaMemcpyAsync(ctx->cself32, c32.data(), sizeof(float) * c32.size(), cudaMemcpyHostToDevice, ctx->stream));
  LCP_CUDA(cudaMemcpyAsync(ctx->cself64t, ct.data(), sizeof(double) * ct.size(), cudaMemcpyHostToDevice, ctx->stream));
  LCP_CUDA(cudaStreamSynchronize(ctx->stream));   // the host copies are freed on return
  return LCP_OK;
}

int self_correction_apply(lcp_ctx* ctx, const double* phi, double* out, int precision) {
  const int n = 3 * ctx->ns;
  if (precision == LCP_MIXED) return block_apply32(ctx, ctx->cself32, phi, out, true);
  dim3 grid((n + 127) / 128, ctx->M);
  ++ctx->nlaunch, k_self64<<<grid, 128, sizeof(double) * n, ctx->stream>>>(n, ctx->M, ctx->cself64t, phi, out);
  LCP_CUDA(cudaGetLastError());
  return LCP_OK;
}
