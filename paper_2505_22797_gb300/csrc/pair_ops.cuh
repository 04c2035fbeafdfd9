// Internal interface of the pair kernels (forward A, adjoint A^T, d/dbeta).
#pragma once

#include "common.cuh"

namespace mpi {

struct ModelH {
    double beta;
    double G[4];
    int n_ch;
    double p[4];
};
struct GridH {
    int nx, ny;
    double x0, y0, dx, dy;
};

// Prepared geometry of one frame (device scratch, filled by prepare_geometry):
//   rw[t]   = (B r_t, B v_t)            B = beta G, one float4/double4 per sample
//   xcol[i] = B (x0 + (i+1/2)dx, 0)     per column
//   yrow[j] = B (0, y0 + (j+1/2)dy)     per row
// so beta G (x_ij - r_t) = xcol[i] + yrow[j] - B r_t.  For a diagonal G the
// second component of xcol and the first of yrow are exactly 0.
template <typename R>
struct Geometry {
    V4<R> *rw;
    V2<R> *xcol;
    V2<R> *yrow;
};

template <typename R>
size_t geometry_bytes(int64_t T, int nx, int ny);
template <typename R>
Geometry<R> geometry_carve(void *base, int64_t T, int nx, int ny);

template <typename R>
int prepare_geometry(const ModelH &m, const GridH &g, int64_t T, const void *r, const void *v,
                     const Geometry<R> &geo, cudaStream_t st);

// Work decomposition of one operator application on one frame.
// `order` (device, nullable): the dispatch order of the work items (block b
// runs item order[b]); see prepare_item_orders.
struct FwdSplit {
    int n_tiles, n_chunks, chunk_rows, rows_staged;
    const int *order = nullptr;
};
struct AdjSplit {
    int tiles_x, tiles_y, n_chunks, chunk_len;
    const int *order = nullptr;
};
FwdSplit forward_split(int64_t T, int nx, int ny, int elem_bytes, int target_items);
AdjSplit adjoint_split(int64_t T, int nx, int ny, int target_items, int elem_bytes);
int default_target_items();  // adjoint and d/dbeta work items per launch
int forward_target_items();  // forward work items per launch
// Column half-width around a sample that can hold a near-FFP pair (forward).
template <typename R>
int near_columns(const ModelH &m, const GridH &g);

// Dispatch orders of the work items of one frame: items whose samples come
// within the asymptotic radius (u < 144) of their voxels cost up to ~1.7x the
// others, so they are dispatched first (stable partition by a bounding-box
// test on the prepared geometry) and the cheap ones fill the end of the
// launch.  The order changes no result: every item writes its own slot.
// Scratch: item_order_bytes; fills fs->order / as->order (either may be NULL).
template <typename R>
size_t item_order_bytes(const FwdSplit *fs, const AdjSplit *as);
template <typename R>
int prepare_item_orders(const GridH &g, int64_t T, const Geometry<R> &geo, FwdSplit *fs,
                        AdjSplit *as, void *scratch, cudaStream_t st);

// Partial-sum scratch sizes (bytes).
template <typename R>
size_t forward_partial_bytes(const FwdSplit &sp, int n_ch, int64_t T);
template <typename R>
size_t adjoint_partial_bytes(const AdjSplit &sp, int nx, int ny);
size_t dbeta_partial_bytes(const AdjSplit &sp);

// One application of A: c (R or double, [ny][nx]) -> s_out ([n_ch][T]); the
// output type is OUT (float or double).  `part` is forward_partial_bytes of
// scratch.  Deterministic.
template <typename R, typename CIN, typename OUT>
int launch_forward(const ModelH &m, const GridH &g, int64_t T, const Geometry<R> &geo,
                   const FwdSplit &sp, const CIN *c, R *part, OUT *s_out, cudaStream_t st);

// One application of A^T: s ([n_ch][T], type R) -> out ([ny][nx], OUT).
// If cg_p != nullptr the epilogue instead writes out = A^T s + nu * cg_p
// (OUT must be double) and partial sums of <cg_p, out> into dot_part
// (adjoint_dot_blocks(nx, ny) of them).
template <typename R, typename OUT>
int launch_adjoint(const ModelH &m, const GridH &g, int64_t T, const Geometry<R> &geo,
                   const AdjSplit &sp, const R *s, R *part, OUT *out, const double *cg_p,
                   const double *nu_dev, double *dot_part, cudaStream_t st);
int adjoint_dot_blocks(int nx, int ny);

// Reduction of per-chunk partial sums (pair operators): out[e] = sum over
// chunks of part[c][e] in a fixed order, FP64.  With cg_p the epilogue writes
// out = sum + nu cg_p (OUT double) and partial sums of <cg_p, out>
// (reduce_dot_blocks(len) of them) into dot_part.
template <typename R, typename OUT>
int reduce_chunks(const R *part, int n_chunks, int64_t len, OUT *out, const double *cg_p,
                  const double *nu_dev, double *dot_part, cudaStream_t st);
int reduce_dot_blocks(int64_t len);

// d/dbeta <g, A(c; beta)>: c [ny][nx] (R), g [n_ch][T] (R) -> *out_dev (FP64).
template <typename R>
int launch_dbeta(const ModelH &m, const GridH &g, int64_t T, const Geometry<R> &geo,
                 const AdjSplit &sp, const R *c, const R *gs, double *part, double *out_dev,
                 cudaStream_t st);

}  // namespace mpi
