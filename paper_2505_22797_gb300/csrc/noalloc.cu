// mpi_forward_noalloc: the forward operator A without any device allocation.
//
// Some callers cannot let a library allocate device memory once they are
// running: acquisition or real-time loops that fix their memory budget at
// start-up so that a long scan can never fail half-way on an allocation,
// applications whose framework owns all device memory through its own pool
// (a raw allocation bypasses its accounting and can fragment it), and code
// that must not risk the implicit device synchronisation of cudaFree.  For
// them this entry point computes exactly what mpi_forward computes, but its
// scratch (the prepared geometry and the per-chunk partial sums) lives in a
// fixed array in device global memory that is part of the library image.
//
// The array is kNoAllocScratchBytes (32 MiB) on every GPU that loads the
// library and stays there until the process exits.  All calls share it and
// it keeps whatever the previous call left in it; this entry point writes
// every byte it later reads, so nothing has to be cleared between calls.
// Calls whose execution overlaps on the GPU (different streams, or different
// host threads, at the same time on the same device) race on the array and
// give wrong results: serialise them.
#include <algorithm>
#include <mutex>

#include "pair_ops.cuh"

namespace mpi {

int check_model(const mpi_model *m);
int check_grid(const mpi_grid_desc *g);
int check_traj(const mpi_traj *t);
int check_dtype(mpi_dtype d);
ModelH to_host(const mpi_model *m);
GridH to_host(const mpi_grid_desc *g);

constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;

// The scratch itself.  In host code this name is only a stand-in for the
// device symbol, never a usable address: the address comes from
// cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_ptr[kMaxDevices] = {};

// Device address of the scratch array for the current device, looked up once
// per device (with that device current) and cached for the life of the
// process.  cudaDeviceReset unloads the device image the address points into,
// so after a reset of a device the cached address is stale: this entry point
// must not be called on a device that has been reset.
int noalloc_scratch(void **out)
{
    int dev = 0;
    MPI_TRY_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("device ordinal %d out of range for the no-allocation scratch", dev);
        return MPI_ERR_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        MPI_TRY_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return MPI_OK;
}

template <typename R>
int forward_noalloc_impl(const ModelH &m, const GridH &g, const mpi_traj *tr, const void *c,
                         void *s, cudaStream_t st)
{
    const int64_t T = tr->T;
    if (T == 0) return MPI_OK;
    auto up = [](size_t b) { return (b + 255) & ~size_t(255); };
    const size_t geo_bytes = up(geometry_bytes<R>(T, g.nx, g.ny));
    const size_t per_chunk = sizeof(R) * size_t(m.n_ch) * size_t(T);
    if (geo_bytes + up(per_chunk) > kNoAllocScratchBytes) {
        set_error("mpi_forward_noalloc: %lld samples on a %d x %d grid need %zu bytes of scratch, "
                  "more than its fixed %zu bytes (about %lld samples with %d channels in %s)",
                  (long long)T, g.nx, g.ny, geo_bytes + up(per_chunk), kNoAllocScratchBytes,
                  (long long)(kNoAllocScratchBytes / (sizeof(V4<R>) + sizeof(R) * m.n_ch)),
                  m.n_ch, sizeof(R) == 4 ? "FP32" : "FP64");
        return MPI_ERR_UNSUPPORTED;
    }
    // As many row chunks as the default split wants, capped by what fits.
    FwdSplit sp = forward_split(T, g.nx, g.ny, sizeof(R), forward_target_items());
    const int max_chunks = (int)std::min<size_t>(
        (kNoAllocScratchBytes - geo_bytes) / up(per_chunk), (size_t)g.ny);
    if (sp.n_chunks > max_chunks)
        sp = forward_split(T, g.nx, g.ny, sizeof(R), sp.n_tiles * std::max(1, max_chunks));
    if ((size_t)sp.n_chunks * per_chunk + geo_bytes > kNoAllocScratchBytes) {
        set_error("mpi_forward_noalloc: internal split does not fit the scratch");
        return MPI_ERR_UNSUPPORTED;
    }

    void *base = nullptr;
    MPI_TRY(noalloc_scratch(&base));
    char *p = static_cast<char *>(base);
    const Geometry<R> geo = geometry_carve<R>(p, T, g.nx, g.ny);
    R *part = reinterpret_cast<R *>(p + geo_bytes);
    MPI_TRY(prepare_geometry<R>(m, g, T, tr->r, tr->v, geo, st));
    return launch_forward<R, R, R>(m, g, T, geo, sp, static_cast<const R *>(c), part,
                                   static_cast<R *>(s), st);
}
}  // namespace

}  // namespace mpi

using namespace mpi;

extern "C" int mpi_forward_noalloc(const mpi_model *model, const mpi_grid_desc *grid,
                                   const mpi_traj *traj, mpi_dtype dtype, const void *c, void *s,
                                   void *stream)
{
    MPI_TRY(check_model(model));
    MPI_TRY(check_grid(grid));
    MPI_TRY(check_traj(traj));
    MPI_TRY(check_dtype(dtype));
    if (traj->T > 0 && (!c || !s)) { set_error("c or s is NULL"); return MPI_ERR_INVALID; }
    const ModelH m = to_host(model);
    const GridH g = to_host(grid);
    return dtype == MPI_F32 ? forward_noalloc_impl<float>(m, g, traj, c, s, as_stream(stream))
                            : forward_noalloc_impl<double>(m, g, traj, c, s, as_stream(stream));
}
