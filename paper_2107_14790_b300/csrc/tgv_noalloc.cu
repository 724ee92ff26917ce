// tgv_energy_noalloc: the energy / dual value / gap reduction for callers that
// must not allocate device memory (see include/tgv.h).  Its scratch is the
// fixed device array below instead of a cudaMalloc'd buffer; everything else
// is the same pair of kernels tgv_energy launches.
#include <mutex>

#include "tgv_internal.cuh"

namespace {

// 3 partial sums per CTA of the energy kernel (a persistent grid of sixteen CTAs per
// SM, whatever the brick count), then the 4 result doubles.  Every GPU that loads
// this library holds it (about 100 KB) until the process exits.
constexpr int64_t kMaxPartials = 4096;
constexpr int64_t kPartialDoubles = 3 * kMaxPartials;
static __device__ __align__(256) double g_noalloc_scratch[kPartialDoubles + 4];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double* g_scratch_addr[kMaxDevices] = {};  // device address of g_noalloc_scratch, per device

// Looks up the array's device address once per device (the current one).  In
// host code the symbol is only a host-side stand-in; the kernels must be
// given the address cudaGetSymbolAddress returns.
tgv_status scratch_for_current_device(double** out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return TGV_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return TGV_ERR_CUDA;
        }
        g_scratch_addr[dev] = (double*)p;
    }
    *out = g_scratch_addr[dev];
    return TGV_OK;
}

}  // namespace

extern "C" tgv_status tgv_energy_noalloc(const tgv_state_view* s, const tgv_params* prm, void* stream, double* out)
{
    if (!s || !prm || !out) return TGV_ERR_INVALID_ARG;
    if (s->nbricks < 0 || s->nall < s->nbricks) return TGV_ERR_INVALID_ARG;
    if (prm->nbins < 2 || prm->nbins > TGV_MAX_BINS) return TGV_ERR_INVALID_ARG;
    if (prm->storage < TGV_STORAGE_FP32 || prm->storage > TGV_STORAGE_FX16) return TGV_ERR_INVALID_ARG;
    if (prm->centres != TGV_CENTRES_ENDPOINTS && prm->centres != TGV_CENTRES_MIDPOINTS) return TGV_ERR_INVALID_ARG;
    if (!(prm->box_v > 0.0f)) return TGV_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (s->nbricks == 0) {
        const double empty[4] = {0.0, 0.0, 0.0, 1.0};
        cudaError_t e = cudaMemcpyAsync(out, empty, sizeof(empty), cudaMemcpyDefault, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        return e == cudaSuccess ? TGV_OK : TGV_ERR_CUDA;
    }
    if (!s->u || !s->v || !s->p || !s->q || !s->hist || !s->nbr) return TGV_ERR_INVALID_ARG;
    if (tgv_energy_grid(s->nbricks) > kMaxPartials) return TGV_ERR_BUDGET;  // a GPU with over 256 SMs
    double* scratch = nullptr;
    tgv_status rc = scratch_for_current_device(&scratch);
    if (rc != TGV_OK) return rc;
    // Each block writes its own partial slot and the reduction writes all four
    // results before anything reads them, so nothing has to be cleared first.
    double* result = scratch + kPartialDoubles;
    cudaError_t e = tgv_launch_energy_view(*s, *prm, st, scratch, result);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, result, 4 * sizeof(double), cudaMemcpyDefault, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return TGV_ERR_CUDA;
    }
    return TGV_OK;
}
