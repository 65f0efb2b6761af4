// Allocation-free variant of the stresslet apply, out = (K + P) phi.
//
// Some callers cannot allocate GPU memory at all: code that runs inside an
// allocator or memory-pool callback, a host that has handed its whole device
// memory budget to another component and forbids further cudaMalloc, or a
// real-time loop where an allocation could block or fail mid-step.  For them
// this file offers one entry point that needs no context and allocates
// nothing: every scratch buffer (quadrature template, Gram inverse, split
// centres, rigid coefficients, FP32 density copy, partial sums) lives in one
// fixed array compiled into the library.  Every GPU that loads the library
// holds that array (LCP_NOALLOC_SCRATCH_BYTES) until the process exits.
//
// The array is shared by all calls and keeps the last call's contents; the
// partial sums, which must start at zero, are cleared by every call.  Calls
// whose GPU work overlaps (different streams or host threads without
// ordering) race on the array and give wrong results: order them.
#include <mutex>

#include "common.cuh"

namespace {

constexpr int NA_MAX_BODIES = 128;
constexpr int NA_MAX_NODES = 16384;
constexpr int NA_MAX_NS = 512;
constexpr int NA_MAX_NT = 256;
constexpr int NA_SLOTS = 4;   // partial-sum slots per target (grid sized to keep within this)

constexpr size_t al(size_t b) { return (b + 255) & ~(size_t)255; }
constexpr size_t OFF_T64 = 0;
constexpr size_t OFF_T32 = OFF_T64 + al(sizeof(double) * 8 * NA_MAX_NS);
constexpr size_t OFF_TN = OFF_T32 + al(sizeof(float) * 6 * NA_MAX_NS);
constexpr size_t OFF_GINV = OFF_TN + al(sizeof(double) * 2 * NA_MAX_NT);
constexpr size_t OFF_C32 = OFF_GINV + al(sizeof(double) * 36);
constexpr size_t OFF_COEF = OFF_C32 + al(sizeof(float) * 8 * NA_MAX_BODIES);
constexpr size_t OFF_PHI32 = OFF_COEF + al(sizeof(double) * 6 * NA_MAX_BODIES);
constexpr size_t OFF_PART = OFF_PHI32 + al(sizeof(float) * 3 * NA_MAX_NODES);
constexpr size_t NA_BYTES = OFF_PART + al(sizeof(double) * 3 * NA_MAX_NODES * NA_SLOTS);

}  // namespace

// The fixed scratch area (about 1.8 MB).
static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

// Device address of the scratch area, looked up once per device and kept for
// the life of the process (a cudaDeviceReset invalidates it; the header tells
// callers not to use this entry point on a device after a reset).
static int scratch_address(int dev, unsigned char** out) {
  static std::mutex mu;
  static unsigned char* addr[64] = {nullptr};
  if (dev < 0 || dev >= 64) return LCP_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) {
      lcp_set_thread_error(std::string("cudaGetSymbolAddress of the scratch area: ") + cudaGetErrorString(e));
      return LCP_ERR_CUDA;
    }
    addr[dev] = (unsigned char*)p;
  }
  *out = addr[dev];
  return LCP_OK;
}

#define NA_CUDA(call)                                                                  \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess) {                                                           \
      lcp_set_thread_error(std::string(#call) + ": " + cudaGetErrorString(e_));        \
      return LCP_ERR_CUDA;                                                             \
    }                                                                                  \
  } while (0)

extern "C" int lcp_stokes_apply_noalloc(int n_bodies, int n_theta, int n_phi, double radius,
                                        const double* centers, const double* phi, double* out, int precision,
                                        void* cuda_stream) {
  const long long ns = (long long)n_theta * n_phi;
  const long long N = ns * n_bodies;
  if (n_bodies < 1 || n_bodies > NA_MAX_BODIES || n_theta < 2 || n_theta > NA_MAX_NT || n_phi < 4 ||
      (n_phi & 1) || ns > NA_MAX_NS || N > NA_MAX_NODES) {
    lcp_set_thread_error("lcp_stokes_apply_noalloc: sizes beyond the fixed scratch area (at most 128 bodies, "
                         "512 nodes per sphere, 16384 nodes in total; n_phi even)");
    return LCP_ERR_INVALID_ARG;
  }
  if (!(radius > 0.0) || !centers || !phi || !out || (precision != LCP_FP64 && precision != LCP_MIXED)) {
    lcp_set_thread_error("lcp_stokes_apply_noalloc: invalid radius, pointer or precision");
    return LCP_ERR_INVALID_ARG;
  }
  int dev = 0;
  NA_CUDA(cudaGetDevice(&dev));
  unsigned char* base = nullptr;
  LCP_TRY(scratch_address(dev, &base));
  cudaStream_t st = (cudaStream_t)cuda_stream;
  double* tmpl64 = (double*)(base + OFF_T64);
  float* tmpl32 = (float*)(base + OFF_T32);
  double* tnodes = (double*)(base + OFF_TN);
  double* ginv = (double*)(base + OFF_GINV);
  float* c32 = (float*)(base + OFF_C32);
  double* coef = (double*)(base + OFF_COEF);
  float* phi32 = (float*)(base + OFF_PHI32);
  double* partial = (double*)(base + OFF_PART);
  const int M = n_bodies, nsi = (int)ns, Ni = (int)N;

  // geometry of this call
  k_template<<<1, 256, 0, st>>>(n_theta, n_phi, radius, tmpl64, tmpl32, tnodes);
  k_gram_inverse<<<1, 32, 0, st>>>(nsi, tmpl64, ginv);
  k_centers32<<<(M + 127) / 128, 128, 0, st>>>(M, centers, c32);
  k_moments<<<(M * 32 + 127) / 128, 128, 0, st>>>(M, nsi, tmpl64, phi, ginv, coef);

  // grid: at most one wave, and few enough CTAs that no target block is
  // shared by more than NA_SLOTS of them
  const int tpb = precision == LCP_MIXED ? PAIR32_TARGETS : PAIR_THREADS_PUBLIC;   // targets per CTA
  const int ntb = (Ni + tpb - 1) / tpb;
  const int units = ntb * M;
  const int ns_pad = (nsi + 3) & ~3;
  const size_t smem = precision == LCP_MIXED
                          ? sizeof(float) * (6 * ns_pad + 3 * PAIR_CHUNK_PUBLIC * ns_pad)
                          : sizeof(double) * (6 * nsi + 3 * PAIR_CHUNK_PUBLIC * nsi);
  int sms = 0, occ = 0;
  NA_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  if (precision == LCP_MIXED) {
    if (smem > 48 * 1024) NA_CUDA(raise_smem_limit((const void*)k_pair32, smem));
    NA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_pair32, PAIR_THREADS_PUBLIC, smem));
  } else {
    if (smem > 48 * 1024) NA_CUDA(raise_smem_limit((const void*)k_pair64, smem));
    NA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_pair64, PAIR_THREADS_PUBLIC, smem));
  }
  const int min_per = (M + NA_SLOTS - 2) / (NA_SLOTS - 1);   // ceil(M / (slots - 1)) units per CTA
  long long grid = (long long)sms * (occ > 0 ? occ : 1);
  if (grid > units / min_per) grid = units / min_per;
  if (grid < 1) grid = 1;
  Units un{units, (int)grid, M};

  NA_CUDA(cudaMemsetAsync(partial, 0, sizeof(double) * 3 * (size_t)Ni * NA_SLOTS, st));
  if (precision == LCP_MIXED) {
    k_to_f32<<<(3 * Ni + 255) / 256, 256, 0, st>>>(3 * Ni, phi, phi32);
    k_pair32<<<(int)grid, PAIR_THREADS_PUBLIC, smem, st>>>(Ni, nsi, ns_pad, un, tmpl32, c32, phi32, partial);
  } else {
    k_pair64<<<(int)grid, PAIR_THREADS_PUBLIC, smem, st>>>(Ni, nsi, un, tmpl64, centers, phi, partial);
  }
  k_finish<<<(Ni + 255) / 256, 256, 0, st>>>(Ni, nsi, NA_SLOTS, partial, coef, tmpl64, out);
  NA_CUDA(cudaGetLastError());
  NA_CUDA(cudaStreamSynchronize(st));
  return LCP_OK;
}
