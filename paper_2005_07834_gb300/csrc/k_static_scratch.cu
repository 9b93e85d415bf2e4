// lrs_solve_w_static: the Dyson solve for W without any device allocation.
//
// Some callers cannot call cudaMalloc: a plugin running inside a host program
// whose caching allocator has already reserved the device memory (a foreign
// cudaMalloc would fail or fragment that pool), a latency-critical loop that
// cannot afford the implicit device synchronisation of cudaMalloc/cudaFree,
// or an embedded caller with a fixed memory budget fixed at start-up.  For
// them this entry point takes every input and output from the caller and
// keeps its scratch (LU matrix, pivots, status words, point radii) in one
// file-scope __device__ array of fixed size.  The array is reserved on a GPU
// when the driver loads this file's module there: with CUDA's default lazy
// module loading that is the first call on that device (at library load with
// CUDA_MODULE_LOADING=EAGER); it is then held until the process exits.
//
// The array is shared by every call on a device and keeps the last call's
// contents; the status words are cleared at the start of each call.  Calls
// that overlap on the GPU (two streams, or two host threads) race on it and
// must be serialised by the caller.  Each call waits for its stream (it reads
// the pivot status back), so a call on a stream that is being captured is
// refused before any work.
#include <mutex>

#include "lrs_internal.h"

namespace lrs {

// Host launchers of k_linalg.cu (external linkage, not part of the internal header).
int dgemm_t(lrs_ctx* ctx, bool ta, bool tb, int m, int n, int k, double alpha, const double* a, int lda,
            const double* ks, const double* b, int ldb, const double* cs, double beta, double* c, int ldc);
int lu_factor(lrs_ctx* ctx, double* A, int n, int* ipiv, int* status);
int lu_solve(lrs_ctx* ctx, const double* LU, int n, const int* ipiv, double* B, int nrhs, int ldb);

namespace {

constexpr size_t kMatBytes = (size_t)LRS_STATIC_MAX_NPTS * LRS_STATIC_MAX_NPTS * sizeof(double);
constexpr size_t kPivBytes = (size_t)LRS_STATIC_MAX_NPTS * sizeof(int);
constexpr size_t kStatusBytes = 256;
constexpr size_t kRadialBytes = (size_t)LRS_STATIC_MAX_NPTS * sizeof(RadialUnit);
constexpr size_t kScratchBytes = kMatBytes + kPivBytes + kStatusBytes + kRadialBytes;
static_assert(kMatBytes % 256 == 0 && kPivBytes % 256 == 0, "scratch sections must stay 256-byte aligned");

static __device__ __align__(256) double g_scratch[kScratchBytes / sizeof(double)];

constexpr int kMaxDevices = 256;
std::mutex g_mutex;
void* g_scratch_addr[kMaxDevices] = {};

__global__ void static_add_identity_kernel(double* __restrict__ a, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[(size_t)i * n + i] += 1.0;
}

// Device address of g_scratch on the current device; looked up once per device.
int scratch_address(int device, char** out) {
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_addr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || p == nullptr)
      return set_error(LRS_ERR_CUDA, "cudaGetSymbolAddress of the static scratch failed: %s",
                       cudaGetErrorString(e));
    g_scratch_addr[device] = p;
  }
  *out = static_cast<char*>(g_scratch_addr[device]);
  return LRS_OK;
}

}  // namespace
}  // namespace lrs

using namespace lrs;

extern "C" int lrs_solve_w_static(int npts, int lmax, const double* pts_dev, const double* wts_dev,
                                  const double* chi0_dev, double* w_dev, void* stream) {
  clear_error();
  if (npts < 1 || npts > LRS_STATIC_MAX_NPTS)
    return set_error(LRS_ERR_ARG, "npts = %d outside [1, %d], the size of the statically reserved scratch",
                     npts, LRS_STATIC_MAX_NPTS);
  if (lmax < 0 || lmax > 64) return set_error(LRS_ERR_ARG, "lmax = %d out of [0,64]", lmax);
  if (!pts_dev || !wts_dev || !chi0_dev || !w_dev) return set_error(LRS_ERR_ARG, "null device pointer");
  cudaStreamCaptureStatus capture = cudaStreamCaptureStatusNone;
  LRS_CUDA_TRY(cudaStreamIsCapturing(static_cast<cudaStream_t>(stream), &capture));
  if (capture != cudaStreamCaptureStatusNone)
    return set_error(LRS_ERR_STATE, "lrs_solve_w_static waits for its stream and cannot run while it is captured");
  int device = -1;
  LRS_CUDA_TRY(cudaGetDevice(&device));
  if (device < 0 || device >= kMaxDevices) return set_error(LRS_ERR_ARG, "device %d not supported", device);
  char* base = nullptr;
  LRS_TRY(scratch_address(device, &base));
  double* A = reinterpret_cast<double*>(base);
  int* ipiv = reinterpret_cast<int*>(base + kMatBytes);
  int* status = reinterpret_cast<int*>(base + kMatBytes + kPivBytes);
  RadialUnit* ru = reinterpret_cast<RadialUnit*>(base + kMatBytes + kPivBytes + kStatusBytes);

  // A context and a site that only point at caller memory and at the static
  // scratch: the launchers below find every buffer already large enough and
  // allocate nothing.
  lrs_ctx ctx;
  ctx.device = device;
  ctx.stream = static_cast<cudaStream_t>(stream);
  ctx.ws.ru.ptr = ru;
  ctx.ws.ru.count = LRS_STATIC_MAX_NPTS;
  Site site;
  site.npts = npts;
  site.lmax = lmax;
  site.pts.ptr = const_cast<double*>(pts_dev);
  site.pts.count = 3 * (size_t)npts;

  const int n = npts;
  LRS_CUDA_TRY(cudaMemsetAsync(status, 0, kStatusBytes, ctx.stream));
  // v into the output buffer; it becomes W after the substitutions
  LRS_TRY(coulomb_build(&ctx, site, w_dev));
  // A = I - (v Q)(chi0 Q)
  LRS_TRY(dgemm_t(&ctx, false, false, n, n, n, -1.0, w_dev, n, wts_dev, chi0_dev, n, wts_dev, 0.0, A, n));
  static_add_identity_kernel<<<(n + 255) / 256, 256, 0, ctx.stream>>>(A, n);
  LRS_TRY(after_launch(&ctx, "static_add_identity_kernel"));
  LRS_TRY(lu_factor(&ctx, A, n, ipiv, status));
  LRS_TRY(lu_solve(&ctx, A, n, ipiv, w_dev, n, n));
  int host_status[2] = {0, 0};
  LRS_CUDA_TRY(cudaMemcpyAsync(host_status, status, sizeof(host_status), cudaMemcpyDeviceToHost, ctx.stream));
  LRS_CUDA_TRY(cudaStreamSynchronize(ctx.stream));
  if (host_status[0] != 0)
    return set_error(LRS_ERR_NUMERIC, "Dyson LU: zero or non-finite pivot in column %d", host_status[1]);
  return LRS_OK;
}
