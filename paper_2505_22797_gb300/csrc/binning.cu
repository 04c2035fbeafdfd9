// Binning of the Core Stage (Eq. first:step): the stable ordering of the
// samples by interpolation cell and the exclusive scans that turn per-cell
// counts into run offsets.  The gather and the transpose walk each cell's
// samples as one contiguous run, in ascending sample order, so every sum of
// the solve has a fixed order.
//
// The ordering is a least-significant-digit radix sort of the cell indices
// (8-bit digits, as many passes as the largest cell index has digits).  Each
// pass is stable, so a cell's samples keep their ascending order and no
// per-cell sort follows.  One pass is three launches: a digit histogram per
// tile of kSortTile samples, an exclusive scan of the histograms in
// digit-major order (the first position of each digit's items of each tile),
// and a scatter that ranks a tile's items of one digit in sample order
// (rounds in order, warps in order, lanes in order).  The scan is a fixed
// reduce-then-scan of three launches: no block waits for another.
#include "grid_common.cuh"

namespace mpi {

namespace {

constexpr int kSortThreads = 256;                      // 8 warps
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortRounds = 8;                         // items per thread and tile
constexpr int kSortTile = kSortThreads * kSortRounds;  // 2048 samples
constexpr int kDigitBits = 8;
constexpr int kDigits = 1 << kDigitBits;
static_assert(kSortThreads == kDigits, "the tile bookkeeping runs one thread per digit");

constexpr int kScanBlock = 1024;  // 32 warps
constexpr int kScanPer = 4;       // consecutive entries per thread
constexpr int kScanTile = kScanBlock * kScanPer;

constexpr unsigned kFull = 0xffffffffu;

inline size_t up256(size_t b) { return (b + 255) & ~size_t(255); }
inline int sort_tiles(int64_t T) { return (int)((T + kSortTile - 1) / kSortTile); }
inline int scan_tiles(int64_t n) { return (int)std::max<int64_t>(1, (n + kScanTile - 1) / kScanTile); }

// Per-tile digit counts, hist[d * n_tiles + tile].  Lanes holding the same
// digit add once (the trajectory keeps consecutive samples in one cell).
__global__ void __launch_bounds__(kSortThreads)
k_digit_hist(const int *__restrict__ key, int64_t n, int shift, int n_tiles, int *__restrict__ hist)
{
    __shared__ int h[kDigits];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t base = int64_t(blockIdx.x) * kSortTile;
#pragma unroll
    for (int r = 0; r < kSortRounds; ++r) {
        const int64_t i = base + r * kSortThreads + threadIdx.x;
        const int d = i < n ? (key[i] >> shift) & (kDigits - 1) : -1;
        const unsigned peers = __match_any_sync(kFull, d);
        if (d >= 0 && lane == __ffs(peers) - 1) atomicAdd(&h[d], __popc(peers));
    }
    __syncthreads();
    hist[int64_t(threadIdx.x) * n_tiles + blockIdx.x] = h[threadIdx.x];
}

// One stable pass: tile b's items of digit d go to pos[d][b], pos[d][b] + 1,
// ... in sample order.  val_in null: the first pass (value = sample index).
// key_out null: the last pass (only the values are kept).  Every position is
// formed from the histogram of the same digits, so it lies in [0, n) whatever
// the keys hold.
__global__ void __launch_bounds__(kSortThreads)
k_digit_scatter(const int *__restrict__ key_in, const int *__restrict__ val_in, int64_t n, int shift,
                int n_tiles, const int *__restrict__ pos, int *__restrict__ key_out,
                int *__restrict__ val_out)
{
    __shared__ int s_next[kDigits];              // next position of each digit for this tile
    __shared__ int s_warp[kSortWarps][kDigits];  // a round's items per warp and digit, then their prefix
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    s_next[threadIdx.x] = pos[int64_t(threadIdx.x) * n_tiles + blockIdx.x];
#pragma unroll
    for (int w = 0; w < kSortWarps; ++w) s_warp[w][threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = int64_t(blockIdx.x) * kSortTile;
    for (int r = 0; r < kSortRounds; ++r) {
        const int64_t i = base + r * kSortThreads + threadIdx.x;
        const bool valid = i < n;
        const int key = valid ? key_in[i] : 0;
        const int val = valid ? (val_in ? val_in[i] : int(i)) : 0;
        const int d = valid ? (key >> shift) & (kDigits - 1) : -1;
        const unsigned peers = __match_any_sync(kFull, d);
        const int rank = __popc(peers & ((1u << lane) - 1u));
        if (valid && rank == 0) s_warp[warp][d] = __popc(peers);
        __syncthreads();
        int run = 0;  // thread = digit: exclusive prefix of the round's counts over the warps
#pragma unroll
        for (int w = 0; w < kSortWarps; ++w) {
            const int c = s_warp[w][threadIdx.x];
            s_warp[w][threadIdx.x] = run;
            run += c;
        }
        __syncthreads();
        if (valid) {
            const int p = s_next[d] + s_warp[warp][d] + rank;
            if (key_out) key_out[p] = key;
            val_out[p] = val;
        }
        __syncthreads();
        s_next[threadIdx.x] += run;
#pragma unroll
        for (int w = 0; w < kSortWarps; ++w) s_warp[w][threadIdx.x] = 0;
        __syncthreads();
    }
}

__global__ void k_iota(int64_t n, int *__restrict__ out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = int(i);
}

// Exclusive scan of one int per thread over a kScanBlock block; *total gets
// the block's sum.  s_w: 32 ints of shared memory.
__device__ __forceinline__ int block_scan_excl(int v, int *s_w, int *total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_w[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int w = s_w[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(kFull, w, o);
            if (lane >= o) w += y;
        }
        s_w[lane] = w;
    }
    __syncthreads();
    *total = s_w[31];
    return (warp ? s_w[warp - 1] : 0) + x - v;
}

// Sum of each tile of kScanTile entries.
__global__ void __launch_bounds__(kScanBlock)
k_scan_reduce(const int *__restrict__ in, int64_t n, int *__restrict__ part)
{
    __shared__ int s_w[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t i0 = int64_t(blockIdx.x) * kScanTile + int64_t(threadIdx.x) * kScanPer;
    int v = 0;
#pragma unroll
    for (int k = 0; k < kScanPer; ++k)
        if (i0 + k < n) v += in[i0 + k];
    v = __reduce_add_sync(kFull, v);
    if (lane == 0) s_w[warp] = v;
    __syncthreads();
    if (warp == 0) {
        const int w = __reduce_add_sync(kFull, s_w[lane]);
        if (lane == 0) part[blockIdx.x] = w;
    }
}

// Exclusive scan of the nb tile sums in place; part[nb] = the total.
__global__ void __launch_bounds__(kScanBlock) k_scan_top(int nb, int *__restrict__ part)
{
    __shared__ int s_w[32];
    const int per = (nb + kScanBlock - 1) / kScanBlock;
    const int b0 = threadIdx.x * per, b1 = min(nb, b0 + per);
    int local = 0;
    for (int k = b0; k < b1; ++k) local += part[k];
    int total;
    int run = block_scan_excl(local, s_w, &total);
    for (int k = b0; k < b1; ++k) {
        const int c = part[k];
        part[k] = run;
        run += c;
    }
    if (threadIdx.x == 0) part[nb] = total;
}

// out[i] = part[tile] + the exclusive prefix of in within the tile; out[n] =
// the total.  in and out are distinct arrays.
__global__ void __launch_bounds__(kScanBlock)
k_scan_tiles(const int *__restrict__ in, int64_t n, const int *__restrict__ part, int nb, int *__restrict__ out)
{
    __shared__ int s_w[32];
    const int64_t i0 = int64_t(blockIdx.x) * kScanTile + int64_t(threadIdx.x) * kScanPer;
    int c[kScanPer];
    int local = 0;
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
        c[k] = i0 + k < n ? in[i0 + k] : 0;
        local += c[k];
    }
    int total;
    int run = part[blockIdx.x] + block_scan_excl(local, s_w, &total);
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
        if (i0 + k < n) out[i0 + k] = run;
        run += c[k];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = part[nb];
}

// count[c] = the number of samples with cell_of[t] = c; values outside
// [0, n_cells) are not counted.
__global__ void k_cell_hist(const int *__restrict__ cell_of, int64_t T, int n_cells, int *__restrict__ count)
{
    for (int64_t t0 = int64_t(blockIdx.x) * blockDim.x; t0 < T; t0 += int64_t(gridDim.x) * blockDim.x) {
        const int64_t t = t0 + threadIdx.x;
        int c = t < T ? cell_of[t] : -1;
        if (c >= n_cells) c = -1;
        warp_count_add(count, c < 0 ? -1 : c);
    }
}

}  // namespace

size_t cell_scan_bytes(int64_t n) { return up256(sizeof(int) * (size_t(scan_tiles(n)) + 1)); }

size_t cell_order_bytes(int64_t T)
{
    const size_t T1 = size_t(std::max<int64_t>(T, 1));
    const int64_t nh = int64_t(kDigits) * std::max(sort_tiles(T), 1);
    return 4 * up256(sizeof(int) * T1) + 2 * up256(sizeof(int) * size_t(nh + 1)) + cell_scan_bytes(nh);
}

int cell_scan_launch(const int *count, int64_t n, int *offset, void *tmp, cudaStream_t st)
{
    if (n <= 0) {
        MPI_TRY_CUDA(cudaMemsetAsync(offset, 0, sizeof(int), st));
        return MPI_OK;
    }
    int *part = static_cast<int *>(tmp);
    const int nb = scan_tiles(n);
    k_scan_reduce<<<nb, kScanBlock, 0, st>>>(count, n, part);
    MPI_CHECK_LAUNCH();
    k_scan_top<<<1, kScanBlock, 0, st>>>(nb, part);
    MPI_CHECK_LAUNCH();
    k_scan_tiles<<<nb, kScanBlock, 0, st>>>(count, n, part, nb, offset);
    MPI_CHECK_LAUNCH();
    return MPI_OK;
}

int cell_order_launch(int64_t T, const int *cell_of, int n_cells, int *list, void *tmp, cudaStream_t st)
{
    if (T <= 0) return MPI_OK;
    const int bits = n_cells > 1 ? 32 - __builtin_clz(unsigned(n_cells - 1)) : 0;
    const int passes = (bits + kDigitBits - 1) / kDigitBits;
    if (passes == 0) {  // one cell: the identity order
        k_iota<<<grid_blocks(T), 256, 0, st>>>(T, list);
        MPI_CHECK_LAUNCH();
        return MPI_OK;
    }
    const size_t T1 = size_t(T);
    const int nt = sort_tiles(T);
    const int64_t nh = int64_t(kDigits) * nt;
    char *p = static_cast<char *>(tmp);
    int *kbuf[2], *vbuf[2];
    for (int k = 0; k < 2; ++k) {
        kbuf[k] = reinterpret_cast<int *>(p); p += up256(sizeof(int) * T1);
        vbuf[k] = reinterpret_cast<int *>(p); p += up256(sizeof(int) * T1);
    }
    int *hist = reinterpret_cast<int *>(p); p += up256(sizeof(int) * size_t(nh + 1));
    int *pos = reinterpret_cast<int *>(p); p += up256(sizeof(int) * size_t(nh + 1));
    const int *kin = cell_of, *vin = nullptr;
    for (int q = 0; q < passes; ++q) {
        const bool last = q == passes - 1;
        int *kout = last ? nullptr : kbuf[q & 1];
        int *vout = last ? list : vbuf[q & 1];
        k_digit_hist<<<nt, kSortThreads, 0, st>>>(kin, T, q * kDigitBits, nt, hist);
        MPI_CHECK_LAUNCH();
        MPI_TRY(cell_scan_launch(hist, nh, pos, p, st));
        k_digit_scatter<<<nt, kSortThreads, 0, st>>>(kin, vin, T, q * kDigitBits, nt, pos, kout, vout);
        MPI_CHECK_LAUNCH();
        kin = kout;
        vin = vout;
    }
    return MPI_OK;
}

}  // namespace mpi

using namespace mpi;

extern "C" int mpi_cell_order(int64_t T, const int *cell_of, int n_cells, int *list, int *offset, void *stream)
{
    if (T < 0 || T >= (int64_t(1) << 31) || n_cells < 1 || (T > 0 && (!cell_of || !list))) {
        set_error("invalid cell ordering arguments (T %lld, n_cells %d)", (long long)T, n_cells);
        return MPI_ERR_INVALID;
    }
    const cudaStream_t st = as_stream(stream);
    Scratch scr(st);
    const size_t o_cnt = scr.reserve(sizeof(int) * size_t(n_cells));
    const size_t o_tmp = scr.reserve(std::max(cell_order_bytes(T), cell_scan_bytes(n_cells)));
    MPI_TRY(scr.allocate());
    if (T > 0) MPI_TRY(cell_order_launch(T, cell_of, n_cells, list, scr.at<char>(o_tmp), st));
    if (offset) {
        int *count = scr.at<int>(o_cnt);
        MPI_TRY_CUDA(cudaMemsetAsync(count, 0, sizeof(int) * size_t(n_cells), st));
        if (T > 0) {
            k_cell_hist<<<grid_blocks(T), 256, 0, st>>>(cell_of, T, n_cells, count);
            MPI_CHECK_LAUNCH();
        }
        MPI_TRY(cell_scan_launch(count, n_cells, offset, scr.at<char>(o_tmp), st));
    }
    return MPI_OK;
}
