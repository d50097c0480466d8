// lub_pairs_build_static: the candidate-pair build without any allocation.
//
// Some callers cannot allocate device memory while they run: a host code
// that owns a fixed device-memory budget and forbids allocation after
// start-up, for instance because cudaMalloc synchronises the whole device
// (stalling its other streams) and may fail mid-run.  They cannot create a
// lub_ctx either, since that allocates.  This entry point runs the same kernels as lub_pairs_build on a
// fixed scratch array that lives in this file as a static __device__ array:
// every GPU that loads the library holds it (LUB_STATIC_SCRATCH_BYTES) until
// the process exits.
//
// Host code cannot use the array's name as a device address (in host code
// it is a stand-in symbol), so the first call on each device looks up the
// device address with cudaGetSymbolAddress, with that device current, and
// caches it.  That first call should therefore come before any stream
// capture.  Every call shares the array and it keeps the previous call's
// contents; the build clears what must start at zero.  Calls whose work
// overlaps on the GPU (two streams at once) race on the array.
#include <mutex>

#include "lub_internal.cuh"

namespace {

constexpr int64_t kMaxParticles = LUB_STATIC_MAX_PARTICLES;
constexpr int64_t kMaxCells = LUB_STATIC_MAX_CELLS;
// cell grid + 5 per-particle int arrays + 2 float4 records + totals/scan/flags
constexpr size_t kBytes = LUB_STATIC_SCRATCH_BYTES;

static __device__ __align__(256) unsigned char g_scratch[kBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void *g_ptr[kMaxDevices] = {};
int g_sms[kMaxDevices] = {};

// once per device, with that device current
int device_setup(int dev, void **ptr, int *sms)
{
    if (dev < 0 || dev >= kMaxDevices) return LUB_ERR_ARG;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) {
            (void)cudaGetLastError();
            return LUB_ERR_CUDA;
        }
        int n = 0;
        e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            return LUB_ERR_CUDA;
        }
        g_sms[dev] = n;
        g_ptr[dev] = p;
    }
    *ptr = g_ptr[dev];
    *sms = g_sms[dev];
    return LUB_OK;
}

}  // namespace

extern "C" int lub_pairs_build_static(const lub_particles *p, const lub_domain *d, const lub_params *prm,
                                      int32_t *pair_i, int32_t *pair_j, int32_t capacity, int32_t *d_count,
                                      void *stream)
{
    if (!p || !d || !prm || !d_count) return LUB_ERR_ARG;
    if (capacity < 0 || (capacity > 0 && (!pair_i || !pair_j))) return LUB_ERR_ARG;
    if (p->n < 0) return LUB_ERR_ARG;
    if (p->batch_offsets) return LUB_ERR_ARG;  // one suspension only
    if ((int64_t)p->n > kMaxParticles) return LUB_ERR_LIMIT;
    if (p->n > 0 && (!p->x || !p->y || !p->z || !p->qw || !p->qx || !p->qy || !p->qz || !p->r_par || !p->r_perp))
        return LUB_ERR_ARG;
    if (!(p->max_semi_axis > 0.0f)) return LUB_ERR_ARG;  // computing it would need scratch and a host sync
    if (d->n_walls < 0 || d->n_walls > 2 || (d->n_walls > 0 && d->periodic[2])) return LUB_ERR_ARG;
    for (int a = 0; a < 3; ++a)
        if (!(d->L[a] > 0.0) || !isfinite(d->L[a])) return LUB_ERR_ARG;
    for (int w = 0; w < d->n_walls; ++w)
        if ((d->wall_dir[w] != 1 && d->wall_dir[w] != -1) || !isfinite(d->wall_z[w])) return LUB_ERR_ARG;
    if (!(prm->list_cutoff >= 0.0) || !isfinite(prm->list_cutoff)) return LUB_ERR_ARG;
    const double range = 2.0 * p->max_semi_axis + prm->list_cutoff;
    for (int a = 0; a < 3; ++a)
        if (d->periodic[a] && !(d->L[a] > 2.0 * range * (1.0 + 1e-6) + 1e-3)) return LUB_ERR_ARG;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        (void)cudaGetLastError();
        return LUB_ERR_CUDA;
    }
    void *scratch = nullptr;
    int sms = 0;
    int rc = device_setup(dev, &scratch, &sms);
    if (rc) return rc;
    if (pairs_scratch_bytes(p->n, kMaxCells) > kBytes) return LUB_ERR_LIMIT;
    return pairs_build_on_scratch(sms, scratch, kBytes, kMaxCells, make_pview(p), make_dview(d), *prm,
                                  p->max_semi_axis, pair_i, pair_j, capacity, d_count, (cudaStream_t)stream);
}
