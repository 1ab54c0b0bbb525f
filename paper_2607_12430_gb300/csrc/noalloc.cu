// noalloc.cu -- an FP64 residual entry point that allocates nothing.
//
// Some callers cannot allocate device memory at the point where they need
// the residual: code running while a stream is being captured into a CUDA
// graph (cudaMalloc is not permitted there), callbacks invoked from inside
// another library's memory-managed region, or real-time loops whose memory
// budget is fixed at start-up.  They cannot create a handle (a handle grows
// its workspace with cudaMalloc on first use), so this entry point takes no
// handle: its only scratch -- the per-block partial sums of |R|^2 and the
// norm -- lives in the file-scope array below, which every GPU that loads
// this library holds until the process exits.
//
// The kernels are the ones sqrtm_step_residual uses; only where their
// scratch lives differs.
#include <string.h>

#include <mutex>

#include "internal.h"
#include "sqrtm_mp_steps.h"

namespace {

// partials of the residual kernel: one per 64 x 64 output tile, so
// n <= 64 * 64 = 4096; plus the final norm
constexpr int kNoallocMaxN = 4096;
constexpr int kNoallocParts = (kNoallocMaxN / 64) * (kNoallocMaxN / 64);

}  // namespace

static __device__ __align__(256) double g_noalloc_scratch[kNoallocParts + 8];

namespace {

constexpr int kMaxDevices = 64;
double *g_scratch_ptr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mu;

// Device address of the scratch array on the current device (looked up once
// per device, with that device current).
int scratch_for_current_device(double **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 7;
    if (dev < 0 || dev >= kMaxDevices) return 7;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return 7;
        g_scratch_ptr[dev] = (double *)p;
    }
    *out = g_scratch_ptr[dev];
    return 0;
}

}  // namespace

extern "C" int sqrtm_step_residual_noalloc(const double *dA, int64_t lda, const double *dX,
                                           int64_t ldx, int64_t n, int e, float *dRhat,
                                           double *norm_host, void *stream)
{
    if (n < 0) return -5;
    if (n > kNoallocMaxN) return -5;
    if (lda < (n > 1 ? n : 1)) return -2;
    if (ldx < (n > 1 ? n : 1)) return -4;
    if (n > 0 && !dA) return -1;
    if (n > 0 && !dX) return -3;
    if (n > 0 && !dRhat) return -7;
    if (n == 0) {
        if (norm_host) *norm_host = 0.0;
        return 0;
    }
    // the partials must fit the array before anything is launched
    const int np = sqm::residual_f64_parts((int)n);
    if (np > kNoallocParts) return -5;
    double *scratch = nullptr;
    if (int rc = scratch_for_current_device(&scratch)) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    int np_launched = 0;
    if (sqm::launch_residual_f64(dA, lda, dX, ldx, (int)n, e, dRhat, (int)n, scratch + 8, &np_launched, s)) return 7;
    if (np_launched != np) return 7;  // the launcher and residual_f64_parts disagree
    if (sqm::launch_sum_partials(scratch + 8, np, scratch, s)) return 7;
    if (norm_host) {
        double v = 0.0;
        if (cudaMemcpyAsync(&v, scratch, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess) return 7;
        if (cudaStreamSynchronize(s) != cudaSuccess) return 7;
        *norm_host = v;
    }
    return 0;
}
