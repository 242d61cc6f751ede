// rich_static.cu -- photon counts and offsets without any device allocation.
//
// Some callers cannot allocate device memory: code running under a framework
// whose pool allocator owns all of the GPU's memory, or a hook inside a
// simulation step that must not make the synchronising cudaMalloc/cudaFree
// calls. For them, rich_photon_counts_static runs the emission's yield and
// scan kernels with their only scratch -- the per-group sums of the scan --
// taken from the fixed array below instead of from a context.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "rich_internal.h"

namespace rich {
void set_global_error(const std::string &msg);
int yield_block_threads();
}  // namespace rich

using namespace rich;

namespace {

// One 256-track scan group per entry: 4096 entries bound a call to
// 4096 * 256 = 1,048,576 tracks. 32 KiB, present on every GPU that loads the
// library until the process exits.
constexpr int kStaticGroups = 4096;
static __device__ __align__(256) unsigned long long g_static_group_sums[kStaticGroups];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
unsigned long long *g_group_sums_addr[kMaxDevices] = {nullptr};

}  // namespace

extern "C" RICH_API rich_status rich_photon_counts_static(const rich_tracks *t,
                                                          const rich_emit_params *prm,
                                                          uint32_t *counts,
                                                          uint64_t *offsets,
                                                          void *stream) {
    const int64_t max_tracks = (int64_t)kStaticGroups * yield_block_threads();
    if (!t || !prm) {
        set_global_error("rich_photon_counts_static: tracks or params is NULL");
        return RICH_ERR_ARG;
    }
    if (t->n < 0 || t->n > max_tracks) {
        set_global_error("rich_photon_counts_static: " + std::to_string(t->n) +
                         " tracks; this entry point handles at most " +
                         std::to_string(max_tracks));
        return RICH_ERR_ARG;
    }
    if (!offsets || (t->n > 0 && (!counts || !t->x || !t->y || !t->z || !t->dx || !t->dy ||
                                  !t->dz || !t->p || !t->mass || !t->length || !t->event))) {
        set_global_error("rich_photon_counts_static: a required array is NULL");
        return RICH_ERR_ARG;
    }
    if (prm->source != RICH_SOURCE_CHERENKOV &&
        (prm->source != RICH_SOURCE_ISOTROPIC || !(prm->yield_per_mm >= 0.f))) {
        set_global_error("rich_photon_counts_static: unknown source or negative yield");
        return RICH_ERR_ARG;
    }
    if (prm->dispersion && (!(prm->disp_a > 0.f) || !(prm->disp_lambda0 > 0.f) ||
                            !(prm->lambda_min > prm->disp_lambda0))) {
        set_global_error("rich_photon_counts_static: dispersion needs disp_a > 0 and "
                         "0 < disp_lambda0 < lambda_min");
        return RICH_ERR_ARG;
    }
    if (!(prm->n_minus_1 >= 0.f) || !(prm->lambda_min > 0.f) ||
        !(prm->lambda_max > prm->lambda_min)) {
        set_global_error("rich_photon_counts_static: need n-1 >= 0 and 0 < lambda_min < lambda_max");
        return RICH_ERR_ARG;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        set_global_error("rich_photon_counts_static: no usable current CUDA device");
        return RICH_ERR_CUDA;
    }
    unsigned long long *sums = nullptr;
    {
        // set-up, once per device with that device current
        std::lock_guard<std::mutex> lock(g_mutex);
        if (!g_group_sums_addr[dev]) {
            void *p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_static_group_sums);
            if (e != cudaSuccess) {
                cudaGetLastError();
                set_global_error(std::string("rich_photon_counts_static: cudaGetSymbolAddress: ") +
                                 cudaGetErrorString(e));
                return RICH_ERR_CUDA;
            }
            g_group_sums_addr[dev] = static_cast<unsigned long long *>(p);
        }
        sums = g_group_sums_addr[dev];
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    if (t->n == 0) {
        e = cudaMemsetAsync(offsets, 0, sizeof(uint64_t), s);
    } else {
        TracksView tv{t->n, t->x, t->y, t->z, t->dx, t->dy, t->dz, t->p, t->mass, t->length,
                      t->event, t->id, t->n_fixed};
        const uint32_t key0 = (uint32_t)prm->seed, key1 = (uint32_t)(prm->seed >> 32);
        // launch_yield clears the group sums this call uses before adding
        const YieldModel model{
            prm->source == RICH_SOURCE_ISOTROPIC ? (double)prm->yield_per_mm : -1.0,
            prm->source == RICH_SOURCE_CHERENKOV && prm->dispersion ? 1 : 0, prm->disp_a,
            prm->disp_lambda0};
        e = launch_yield(tv, (double)prm->n_minus_1, prm->lambda_min, prm->lambda_max, key0, key1,
                         nullptr, nullptr, counts, sums, s, model);
        if (e == cudaSuccess) e = launch_offsets(counts, sums, t->n, offsets, nullptr, s);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_global_error(std::string("rich_photon_counts_static: ") + cudaGetErrorString(e));
        return RICH_ERR_CUDA;
    }
    return RICH_OK;
}
