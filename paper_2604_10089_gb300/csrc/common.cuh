// Shared device helpers and the internal context of the collision-resolution
// library.  Everything here is GPU-side infrastructure; the arithmetic of the
// method lives in the kernels of the other translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "lcp_gb300.h"

#define LCP_PI 3.14159265358979323846


// ------------------------------------------------------------ reductions
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sumf(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum in a fixed order (deterministic).  `red` must hold
// blockDim.x / 32 doubles.  Every thread receives the result.
__device__ __forceinline__ double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double t = 0.0;
  if (wid == 0) {
    t = lane < nw ? red[lane] : 0.0;
    t = warp_sum(t);
    if (lane == 0) red[0] = t;
  }
  __syncthreads();
  t = red[0];
  __syncthreads();
  return t;
}

// Work decomposition shared by both pair kernels.  The N x N pair sum is cut
// into units (target block tb, source body j); the U = ntb * M units are dealt
// out in contiguous, equal ranges to a grid of G CTAs sized to one full wave
// (SMs x resident CTAs per SM), so no CTA waits for a second wave.  A CTA
// writes one partial per target block it touches into slot
// (c - first CTA touching tb); the finishing kernel sums the slots in order.
struct Units {
  int U, G, M;
  __device__ __forceinline__ int start(int c) const { return (int)(((long long)c * U) / G); }
  __device__ __forceinline__ int first_cta(int tb) const {
    const int u = tb * M;
    int c = (int)(((long long)u * G) / U);
    while (c + 1 < G && start(c + 1) <= u) c++;
    while (c > 0 && start(c) > u) c--;
    return c;
  }
};

// Pair-sum and projection kernels (stokes.cu), launchable from other files.
__global__ void k_pair32(int N, int ns, int ns_pad, Units un, const float* __restrict__ tmpl32,
                         const float* __restrict__ c32, const float* __restrict__ phi32, double* __restrict__ partial);
__global__ void k_pair64(int N, int ns, Units un, const double* __restrict__ tmpl64,
                         const double* __restrict__ centers, const double* __restrict__ phi,
                         double* __restrict__ partial);
__global__ void k_moments(int M, int ns, const double* __restrict__ tmpl64, const double* __restrict__ phi,
                          const double* __restrict__ ginv, double* __restrict__ coef);
__global__ void k_finish(int N, int ns, int splits, const double* __restrict__ partial,
                         const double* __restrict__ coef, const double* __restrict__ tmpl64,
                         double* __restrict__ out);
__global__ void k_to_f32(int L, const double* __restrict__ x, float* __restrict__ y);
// Quadrature template and rigid Gram inverse (geometry.cu).
__global__ void k_template(int nt, int np, double a, double* tmpl64, float* tmpl32, double* tnodes);
__global__ void k_gram_inverse(int ns, const double* tmpl64, double* ginv);
__global__ void k_centers32(int M, const double* c, float* c32);
constexpr int PAIR_THREADS_PUBLIC = 256;     // block size of the pair kernels
constexpr int PAIR32_TARGETS = 512;          // targets per CTA of the FP32 pair kernel (2 per thread)
constexpr int PAIR_CHUNK_PUBLIC = 8;         // source bodies staged per tile
void lcp_set_thread_error(const std::string& msg);

// ------------------------------------------------------------ host side
struct GmresWork;

struct PqnDev {   // quasi-Newton state of one PQN run, all device pointers
  int n, rmax;
  double *x, *g, *p, *Ap, *xt, *xh, *extra, *lop;   // [n]
  double *S, *Y, *U, *V;                             // [rmax][n]
  double *UU, *UV, *VV;                              // [rmax][rmax]
  int* r;                                            // pairs held
  double* scal;                                      // scalar slots (see pqn.cu)
};

struct lcp_ctx {
  lcp_config cfg;
  cudaStream_t stream = nullptr;
  int M = 0, ns = 0, N = 0, n = 0;
  // geometry
  double* tmpl64 = nullptr;   // [ns][8]: xi(3), wn(3) = -(3/4pi) w n, w, 0
  float* tmpl32 = nullptr;    // SoA [6][ns]: xi x,y,z, wn x,y,z
  double* ginv = nullptr;     // [36] inverse Gram matrix of the rigid modes
  double* centers = nullptr;  // [M][3]
  float* centers32 = nullptr; // [M][8]: hi(3), pad, lo(3), pad
  double* axes = nullptr;     // [M][3]
  bool has_axes = false;
  // contacts
  int *ci = nullptr, *cj = nullptr;
  double *cnrm = nullptr, *gap = nullptr, *b = nullptr;
  int *bc_ptr = nullptr, *bc_idx = nullptr;
  int *flags = nullptr, *csr_cnt = nullptr;
  double* U_nc = nullptr;     // [M][6]
  double* phi_unc = nullptr;  // [3N]: density of the last slip solve (warm start along a trajectory)
  bool phi_unc_valid = false;
  int unc_its = 0, unc_warm = 0;   // GMRES iterations / warm start of the last slip solve
  // warm start of the next LCP solve along a trajectory (cfg.warm_start): the last
  // solution and its contact pairs, carried onto the next step's contacts
  double *x_prev = nullptr, *x_warm = nullptr;   // [pair_cap]
  int *ci_prev = nullptr, *cj_prev = nullptr;    // [pair_cap]
  bool x_warm_valid = false;
  double* MDx = nullptr;      // [M][6] collisional velocities M D x of the last solve
  double *cnext = nullptr, *anext = nullptr;   // [M][3] advanced centres / axes
  bool have_solution = false;
  // mobility solve workspace
  int m = 0, splits = 1;
  int num_sms = 0, occ32 = 0, occ64 = 0, occdf = 0;   // pair-kernel grid sizing
  int occ32v[8] = {0};        // occupancy of each FP32 kernel variant
  int v32 = 0;                // FP32 kernel variant in use (autotuned per size class)
  bool sym = true;            // FP32 sums by the symmetric kernel (stokes_sym.cu)
  int sym_v = 0;              // symmetric kernel variant in use
  int sym_ntb = 0, sym_units = 0, sym_slots = 0;   // sym_slots: largest over the variants
  int symv_occ[16] = {0}, symv_grid[16] = {0}, symv_slots[16] = {0};
  std::vector<float4> sym_tparam;  // launch-parameter copy of the source template (duplicated pairs)
  int symdf_grid = 0, symdf_slots = 0;   // the symmetric double-float kernel (stokes_sym_df.cu)
  int* sym_off = nullptr;          // [ntb + 1] first unit of each target block
  long long* sym_roff = nullptr;   // [ntb + 1] first float of each block's reverse rows
  long long* sym_rbase = nullptr;  // [ntb + 1] roff[tb] - (first body + 1) * 3 ns: row of body i at + i * 3 ns
  float* sym_rev = nullptr;        // reverse partial sums, one row per unit (FP32, or (hi, lo) pairs)
  double *V = nullptr, *H = nullptr;  // Krylov basis [(m+1)][3N], Hessenberg etc.
  double* Z = nullptr;                 // preconditioned basis [m][3N] (flexible GMRES)
  float* pinv = nullptr;               // isolated-sphere inverse (3 ns x 3 ns, FP32)
  float* cself32 = nullptr;            // self-interaction correction (3 ns x 3 ns, FP32, row-major)
  double* cself64t = nullptr;          // the same in FP64, transposed
  float* ppart = nullptr;              // split-k partial products of the preconditioner GEMM
  double *phi = nullptr, *rhs = nullptr, *res = nullptr, *wv = nullptr, *dphi = nullptr;
  float* phi32 = nullptr;
  float* phidf = nullptr;     // [N][6] double-FP32 density (hi xyz, lo xyz)
  double* partial = nullptr;  // [splits][N][3]
  double* coef = nullptr;     // [M][6]
  double* dotp = nullptr;     // dot-product partials
  double* FT = nullptr;       // [M][6]
  double* UO = nullptr;       // [M][6]
  double* dscal = nullptr;    // device scalars
  double* hscal = nullptr;    // pinned host mirror
  int dot_blocks = 0;
  // PQN
  PqnDev pq_outer{}, pq_inner{};
  double *Uh = nullptr, *Vh = nullptr;   // Bi-PQN high-fidelity corrections [kmax][n]
  int nh = 0;
  double *tmp_n = nullptr, *tmp_n2 = nullptr, *tmp_n3 = nullptr;
  std::vector<void*> allocs;
  size_t bytes = 0;           // device bytes held (footprint for admission)
  int device = 0;
  bool owns_stream = false;
  // contact-sized buffers live in one arena, re-created when n outgrows it
  void* arena = nullptr;
  size_t arena_bytes = 0;
  int ncap = 0;
  int pair_cap = 0;   // capacity of ci/cj/cnrm/gap
  // kernel timing (lcp_profile)
  bool prof = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<int> ev_kind;
  std::string err;
  unsigned long long nlaunch = 0;   // kernels launched by this context
  // captured CUDA graphs of the GMRES Arnoldi step, one per (column j,
  // operator precision); re-captured when the FP32 kernel variant changes
  struct ArnoldiGraph {
    cudaGraphExec_t exec = nullptr;
    int stamp = -1;
    unsigned long long kernels = 0;
    int c32 = 0, c64 = 0, cdf = 0;
    std::vector<cudaEvent_t> ev;   // timed graphs: event pairs recorded by the graph's own nodes
    std::vector<int> ev_kind;
  };
  std::vector<ArnoldiGraph> agraphs;
  // kernel timing inside graphs: while a timed graph is captured, prof_begin /
  // prof_end record external events into it (cap_ev, cap_kind); after each
  // replay and the host's synchronisation the pairs are read into prof_ms /
  // prof_n (per kind) before the same graph can run again
  std::vector<cudaEvent_t>* cap_ev = nullptr;
  std::vector<int>* cap_kind = nullptr;
  int timed_key = -1;                 // graph replayed last with events to read
  double prof_ms[8] = {0};
  int prof_n[8] = {0};
  // low-fidelity coarse-grid context (Bi-PQN, cfg.lowfi_n_theta > 0): same
  // bodies and stream, no contacts; its mobility solves run FP32 GMRES only
  lcp_ctx* lo = nullptr;
  bool fp32_only = false;
  // reuse across the mobility solves of one configuration: up to rc_max pairs
  // (psi_k, w_k), w_k ~= (K + P) psi_k, the w_k orthonormal, in slots [0, rc_count)
  double* rc_psi = nullptr;   // [rc_max][3N]
  double* rc_w = nullptr;     // [rc_max][3N]
  double* rc_h = nullptr;     // [3 rc_max] projection / Gram-Schmidt coefficients
  double* rc_phi0 = nullptr;  // [3N] start of the current solve, then its direction
  double* rc_r0 = nullptr;    // [3N] start residual of the current solve, then its image
  int rc_max = 0, rc_count = 0;
  // counters of the current solve
  int c_gmres = 0, c_fp64 = 0, c_fp32 = 0, c_df64 = 0;
  int c_recycled = 0;         // solves started from the projection
  // since set-up (never reset): mobility solves, their GMRES iterations, projected starts
  long long tot_solves = 0, tot_gmres = 0, tot_recycled = 0;
};

#define LCP_CUDA(call)                                                            \
  do {                                                                            \
    cudaError_t e_ = (call);                                                      \
    if (e_ != cudaSuccess) {                                                      \
      ctx->err = std::string(#call) + ": " + cudaGetErrorString(e_);              \
      return LCP_ERR_CUDA;                                                        \
    }                                                                             \
  } while (0)

#define LCP_TRY(expr)                  \
  do {                                 \
    int s_ = (expr);                   \
    if (s_ != LCP_OK) return s_;       \
  } while (0)

// Event timing of a launch (lcp_profile): returns the start event or null.
// Inside a graph capture the events are external (recorded by graph nodes at
// every replay) and belong to the graph.
inline cudaEvent_t prof_begin(lcp_ctx* ctx) {
  if (!ctx->prof) return nullptr;
  cudaEvent_t e;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  if (ctx->cap_ev)
    cudaEventRecordWithFlags(e, ctx->stream, cudaEventRecordExternal);
  else
    cudaEventRecord(e, ctx->stream);
  return e;
}
inline void prof_end(lcp_ctx* ctx, cudaEvent_t start, int kind) {
  if (!start) return;
  cudaEvent_t e;
  if (cudaEventCreate(&e) != cudaSuccess) return;
  if (ctx->cap_ev) {
    cudaEventRecordWithFlags(e, ctx->stream, cudaEventRecordExternal);
    ctx->cap_ev->push_back(start);
    ctx->cap_ev->push_back(e);
    ctx->cap_kind->push_back(kind);
    return;
  }
  cudaEventRecord(e, ctx->stream);
  ctx->ev_pool.push_back(start);
  ctx->ev_pool.push_back(e);
  ctx->ev_kind.push_back(kind);
}

// Internal launch helpers implemented in the .cu files.
int geometry_build(lcp_ctx* ctx);
int geometry_update(lcp_ctx* ctx);
int contacts_detect(lcp_ctx* ctx, int* n_out);
int contacts_upload(lcp_ctx* ctx, int n, const lcp_contact* c);
int contacts_csr(lcp_ctx* ctx);
int contacts_carry(lcp_ctx* ctx, int n_prev);   // x_warm from x_prev by body pair
int stokes_apply(lcp_ctx* ctx, const double* phi, double* out, int precision);
int stokes_rhs(lcp_ctx* ctx, const double* FT, int include_slip, double* rhs);
int stokes_coefs(lcp_ctx* ctx, const double* phi, double* coef);
int mobility_solve(lcp_ctx* ctx, const double* FT, int include_slip, double* UO, const double* phi0 = nullptr);
void recycle_reset(lcp_ctx* ctx);   // forget the kept solve pairs (this context and its coarse grid)
int precond_build(lcp_ctx* ctx);
int precond_apply(lcp_ctx* ctx, const double* v, double* z);
int block_apply_reserve(lcp_ctx* ctx);
int block_apply32(lcp_ctx* ctx, const float* mat, const double* v, double* z, bool accumulate);
int self_correction_build(lcp_ctx* ctx);
int self_correction_apply(lcp_ctx* ctx, const double* phi, double* out, int precision);
int scatter_D(lcp_ctx* ctx, const double* x, double* FT);
int gather_Dt(lcp_ctx* ctx, const double* UO, double* out, const double* add);
int rpy_apply(lcp_ctx* ctx, const double* FT, double* UO);
int mvp_high(lcp_ctx* ctx, const double* x, double* Ax);
int mvp_low(lcp_ctx* ctx, const double* x, double* Ax);       // the configured low fidelity
int mvp_rpy(lcp_ctx* ctx, const double* x, double* Ax);       // D^T M_RPY D x
int mvp_lowbie(lcp_ctx* ctx, const double* x, double* Ax);    // D^T M_coarse D x
size_t pqn_bytes(int n, int rmax);
char* pqn_carve(PqnDev* pq, char* base, int n, int rmax);
int pqn_reset(lcp_ctx* ctx, PqnDev* pq);
int lcp_solve_device(lcp_ctx* ctx, int method, double tol, const double* x0, double* x, lcp_stats* st);
void* ctx_alloc(lcp_ctx* ctx, size_t bytes);
// Raises a kernel's dynamic shared-memory limit on the current device to at
// least `bytes` and never lowers it: contexts of different sizes share the
// kernels, and a smaller context set up after a larger one must not cut the
// limit below the larger one's launches.  Thread-safe.
cudaError_t raise_smem_limit(const void* kernel, size_t bytes);
