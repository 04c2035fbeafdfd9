// Device kernels of the pair sums (forward A, adjoint A^T, d/dbeta).
//
// Every (voxel, sample) pair evaluates the Langevin kernel once; there is no
// contraction to hand to the tensor cores (one FMA per pair per channel), so
// the kernels are bound by instruction issue on the FP32 and MUFU (XU) pipes.
// A pair costs the full closed form (3 MUFU: rsqrt, exp2, rcp, and ~18 FP32
// operations) only near the samples; far from them (z >= 12, most pairs) the
// asymptotic form needs one rsqrt and 12 (forward) or 9 (adjoint) FP32
// operations, and within z < 1 the Taylor series replaces the closed form.
// The regime is decided for warp-uniform segments (forward: column ranges of
// a staged row; adjoint: groups of 32 staged samples, or single samples in
// mixed groups); only the near-series check takes a per-pair warp vote.
//
// Both kernels take a frame table by value, so one launch can cover many
// frames of different sizes: blockIdx.x enumerates work items of all frames
// (frame f owns items [item0_f, item0_f + n_items_f)).
#pragma once

#include <algorithm>

#include "langevin.cuh"
#include "pair_ops.cuh"

namespace mpi {

constexpr int kFwdThreads = 128;
#ifndef MPI_FWD_S
#define MPI_FWD_S 2
#endif
constexpr int kFwdS = MPI_FWD_S;  // samples per thread
constexpr int kFwdTile = kFwdThreads * kFwdS;
// Staging of the forward's concentration rows: one copy per block, or (with
// MPI_FWD_WSTAGE) one per warp, so that the warps of a block never wait for
// one another at a barrier (their samples lie in different regimes and
// finish their rows at different times).  A block's row buffers share one
// byte budget.
#ifndef MPI_FWD_WSTAGE
#define MPI_FWD_WSTAGE 0
#endif
constexpr int kFwdStageCopies = MPI_FWD_WSTAGE ? kFwdThreads / 32 : 1;
constexpr size_t kFwdRowBudget = 16 * 1024;
// Rows staged at a time for rows of nx values of elem bytes.
inline int fwd_rows_staged(int chunk_rows, int nx, int elem)
{
    const size_t per = kFwdRowBudget / kFwdStageCopies / (2 * size_t(elem) * size_t(nx));
    return (int)std::max<size_t>(1, std::min<size_t>(size_t(chunk_rows), per));
}
// Dynamic shared memory of a forward block: xcol [nx] and, per copy, yrow [RB]
// and RB rows of (x_i, c_i) pairs.
inline size_t fwd_smem_bytes(int nx, int RB, int elem)
{
    return 2 * size_t(elem) * (size_t(nx) + kFwdStageCopies * (size_t(RB) + size_t(RB) * size_t(nx)));
}

// Warps per adjoint block, and how the staged samples are shared: one copy
// per block (MPI_ADJ_WSTAGE 0, block barriers around the staging) or one per
// warp (1: the warps never wait for one another).  Timed on GB300 at
// 128 x 128 / 65 536 samples: 4 warps with one copy per block 0.453 ms, one
// copy per warp 0.466 ms, 2 warps 0.457 ms, 1 warp 0.537 ms (512 x 512 /
// 2^20 samples: one copy per block 101 ms, per warp 108 ms).
#ifndef MPI_ADJ_WARPS
#define MPI_ADJ_WARPS 4
#endif
#ifndef MPI_ADJ_WSTAGE
#define MPI_ADJ_WSTAGE 0
#endif
constexpr int kAdjStageCopies = MPI_ADJ_WSTAGE ? MPI_ADJ_WARPS : 1;
constexpr int kAdjWarps = MPI_ADJ_WARPS;
constexpr int kAdjThreads = 32 * kAdjWarps;
#ifndef MPI_ADJ_V
#define MPI_ADJ_V 8
#endif
// Tuning knobs (compile time), chosen by timing variants on GB300: minimum
// resident blocks per SM requested from the register allocator for the FP32
// kernels (forward: 6 x 128 threads, 80 registers; adjoint: 5 x 128, 96
// registers -- its packed asymptotic tier spills at 80; at 128 x 128 /
// 65 536 samples 0.431 ms against 0.438 ms with 4 blocks and 0.441 ms with
// 6), and the unroll depth of the forward column loop (packed asymptotic
// loop: 8 columns in flight, 0.457 ms at 128 x 128 / 65 536 samples against
// 0.461 ms with 4 and 0.471 ms with 2).  The FP64 kernels request 2 blocks
// per SM (no spills).
#ifndef MPI_FWD_MINB
#define MPI_FWD_MINB 6
#endif
#ifndef MPI_ADJ_MINB
#define MPI_ADJ_MINB (20 / MPI_ADJ_WARPS)
#endif
#ifndef MPI_FWD_UNROLL
#define MPI_FWD_UNROLL 8
#endif
constexpr int kFwdUnroll = MPI_FWD_UNROLL;
#ifndef MPI_FWD_PACK
#define MPI_FWD_PACK 1
#endif
// A warp's samples as one consecutive run of the trajectory (1: 0.451 ms
// at 128 x 128 / 65 536 samples against 0.456 ms with the block's samples
// interleaved across its warps).
#ifndef MPI_FWD_WARP_RUN
#define MPI_FWD_WARP_RUN 1
#endif
constexpr bool kFwdPack = MPI_FWD_PACK != 0;
// Unroll depth of the full closed-form column loops (a few percent of the
// pairs once the asymptotic tier takes the rest: kept short for code size).
#ifndef MPI_FWD_UNROLL_FAR
#define MPI_FWD_UNROLL_FAR 2
#endif
constexpr int kFwdUnrollFar = MPI_FWD_UNROLL_FAR;
constexpr int kAdjV = MPI_ADJ_V;  // voxels (rows) per thread
constexpr int kAdjTileX = 32;
constexpr int kAdjTileY = kAdjWarps * kAdjV;
#ifndef MPI_ADJ_BLOCK
#define MPI_ADJ_BLOCK 256
#endif
// Unroll depth of the adjoint's asymptotic loop over a group's 32 samples
// (packed: 16 sample pairs; 4 pairs in flight timed fastest, 0.431 ms at
// 128 x 128 / 65 536 samples against 0.432 ms with 1).
#ifndef MPI_ADJ_UNROLL_VFAR
#define MPI_ADJ_UNROLL_VFAR 4
#endif
constexpr int kAdjUnrollVfar = MPI_ADJ_UNROLL_VFAR;
// FP32 asymptotic tier of the adjoint in packed two-lane FP32 arithmetic
// (fma.rn.f32x2 and its add/mul forms, sm_100 and later): the pair term is
// issue-bound, and a packed instruction does two lanes' FP32 work in one
// issue slot (measured on GB300: 126 FP32 FMAs per SM per clock either way,
// from half the instructions).  The staged samples are then also kept as
// even/odd pairs, and each voxel accumulates its even and odd samples in the
// two lanes of a pair (added into the voxel's sum after each group of 32).
#ifndef MPI_ADJ_PACK
#define MPI_ADJ_PACK 1
#endif
constexpr bool kAdjPack = MPI_ADJ_PACK != 0;
// Warp box of the adjoint's regime test: 16 x 16 voxels (1) or 32 x 8 (0).
// The squarer box sends fewer 32-sample groups to the closed form (7.9 %
// against 9.4 % of the groups at 128 x 128 / 65 536 samples): 0.426 ms
// against 0.431 ms there.
#ifndef MPI_ADJ_BOX16
#define MPI_ADJ_BOX16 1
#endif

constexpr int kAdjBlock = MPI_ADJ_BLOCK;  // samples staged per shared-memory block

template <typename R>
struct PairFrame {
    const V4<R> *rw;
    const V2<R> *xcol;
    const V2<R> *yrow;
    const void *in;   // forward: c [ny][nx]; adjoint: s [n_ch][T]; dbeta: c
    const void *in2;  // dbeta: g [n_ch][T]
    void *part;       // partial sums
    int64_t T;
    int64_t item0;
    int nx, ny;
    int n_ch;
    int n_tiles;      // forward: sample tiles; adjoint: voxel tiles
    int tiles_x;      // adjoint only
    int chunk;        // forward: rows per chunk; adjoint: samples per chunk
    int rows_staged;  // forward: rows per shared-memory block
    int near_cols;    // forward: column half-width that can hold a near pair
    int diag;         // G is diagonal (selects the kernel branch in mixed batches)
    const int *order; // nullable: local item index dispatched by local block index
    R p[4];
};

template <typename R, int MAXF>
struct PairBatch {
    int n_frames;
    PairFrame<R> f[MAXF];
};

#ifdef __CUDACC__

template <typename R, int MAXF>
__device__ __forceinline__ int find_frame(const PairBatch<R, MAXF> &B, int64_t item)
{
    int f = 0;
#pragma unroll 1
    for (int q = 1; q < B.n_frames; ++q)
        if (item >= B.f[q].item0) f = q;
    return f;
}

// ---------------------------------------------------------------------------
// One staged row of the forward sum for this thread's samples (diagonal G):
// sa += c a, vx += f y_x, fy += f with f = c d (y.W).  With CLAMP the
// Langevin scalars are evaluated at max(u, near_u), valid for the closed form.
template <typename R, bool CLAMP>
__device__ __forceinline__ void fwd_row_far(int i0, int i1, const V2<R> *__restrict__ xc,
                                            const R (&Rx)[kFwdS],
                                            const R (&yy2)[kFwdS], const R (&Wx)[kFwdS],
                                            const R (&yyW)[kFwdS], R (&sa)[kFwdS], R (&vx)[kFwdS],
                                            R (&fy)[kFwdS])
{
#pragma unroll kFwdUnrollFar
    for (int i = i0; i < i1; ++i) {
        const V2<R> q = xc[i];  // (x_i, c_i) in one load
        const R xi = q.x, ci = q.y;
#pragma unroll
        for (int s = 0; s < kFwdS; ++s) {
            const R yx = xi - Rx[s];
            R u = fmx(yx, yx, yy2[s]);
            if (CLAMP) u = max(u, Lang<R>::near_u);
            R a, d;
            lang_far<R, false>(u, a, d);
            sa[s] = fmx(ci, a, sa[s]);
            const R f = ci * d * fmx(yx, Wx[s], yyW[s]);
            vx[s] = fmx(f, yx, vx[s]);
            fy[s] += f;
        }
    }
}

// The same sums over columns [i0, i1) whose pairs all have u >= vfar_u: the
// asymptotic closed form (one rsqrt per pair).  FP32 with two samples per
// thread and kFwdPack: the two samples are the two lanes of packed FP32
// arithmetic (f32x2, sm_100 and later: the same FP32 work from half the
// issue slots; the FMA pipe then bounds the loop).
template <typename R>
__device__ __forceinline__ void fwd_row_vfar(int i0, int i1, const V2<R> *__restrict__ xc,
                                             const R (&Rx)[kFwdS], const R (&yy2)[kFwdS],
                                             const R (&Wx)[kFwdS], const R (&yyW)[kFwdS],
                                             R (&sa)[kFwdS], R (&vx)[kFwdS], R (&fy)[kFwdS])
{
    if constexpr (kFwdPack && sizeof(R) == 4 && kFwdS == 2) {
        const float2 m1 = make_float2(-1.0f, -1.0f);
        const float2 nRx = make_float2(-Rx[0], -Rx[1]), yy2p = make_float2(yy2[0], yy2[1]);
        const float2 Wxp = make_float2(Wx[0], Wx[1]), yyWp = make_float2(yyW[0], yyW[1]);
        float2 sa2 = make_float2(0.0f, 0.0f), vx2 = sa2, fy2 = sa2;
#pragma unroll kFwdUnroll
        for (int i = i0; i < i1; ++i) {
            const V2<R> q = xc[i];
            const float2 cc = make_float2(q.y, q.y);
            const float2 yx = __fadd2_rn(make_float2(q.x, q.x), nRx);
            const float2 u = __ffma2_rn(yx, yx, yy2p);
            const float2 iz = make_float2(Lang<float>::iz_vfar(u.x), Lang<float>::iz_vfar(u.y));
            const float2 iz2 = __fmul2_rn(iz, iz);
            const float2 a = __ffma2_rn(iz2, m1, iz);                       // iz - iz^2
            const float2 d = __fmul2_rn(__ffma2_rn(a, m1, iz2), iz2);       // (2 iz^2 - iz) iz^2
            sa2 = __ffma2_rn(cc, a, sa2);
            const float2 f = __fmul2_rn(__fmul2_rn(cc, d), __ffma2_rn(yx, Wxp, yyWp));
            vx2 = __ffma2_rn(f, yx, vx2);
            fy2 = __fadd2_rn(fy2, f);
        }
        sa[0] += sa2.x; sa[1] += sa2.y;
        vx[0] += vx2.x; vx[1] += vx2.y;
        fy[0] += fy2.x; fy[1] += fy2.y;
        return;
    }
#pragma unroll kFwdUnroll
    for (int i = i0; i < i1; ++i) {
        const V2<R> q = xc[i];
        const R xi = q.x, ci = q.y;
#pragma unroll
        for (int s = 0; s < kFwdS; ++s) {
            const R yx = xi - Rx[s];
            const R u = fmx(yx, yx, yy2[s]);
            R a, d;
            Lang<R>::ad_vfar(u, a, d);
            sa[s] = fmx(ci, a, sa[s]);
            const R f = ci * d * fmx(yx, Wx[s], yyW[s]);
            vx[s] = fmx(f, yx, vx[s]);
            fy[s] += f;
        }
    }
}

// Replace, for the pairs of one sample on one row with u < near_u, the clamped
// closed-form values (A1, D1) by the Taylor series.  Only columns within
// `win` of the sample's nearest column can qualify (xcol is linear in i).
template <typename R>
__device__ __forceinline__ void fwd_near_fix(int nx, const V2<R> *__restrict__ xc, R Rx, R yy2,
                                             R Wx, R yyW,
                                             R A1, R D1, int win, R &sa, R &vx, R &fy)
{
    const R x0 = xc[0].x;
    const R step = nx > 1 ? xc[1].x - x0 : R(1);
    R fi = (Rx - x0) / step;
    fi = min(max(fi, R(-2 * win - 2)), R(nx + 2 * win + 2));
    const int ic = (int)rint(fi);
    const int i0 = max(0, ic - win), i1 = min(nx - 1, ic + win);
    for (int i = i0; i <= i1; ++i) {
        const R yx = xc[i].x - Rx;
        const R u = fmx(yx, yx, yy2);
        if (u < Lang<R>::near_u) {
            R a, d;
            Lang<R>::ad_near(u, a, d);
            const R ci = xc[i].y;
            sa = fmx(ci, a - A1, sa);
            const R f = ci * (d - D1) * fmx(yx, Wx, yyW);
            vx = fmx(f, yx, vx);
            fy += f;
        }
    }
}

// ---------------------------------------------------------------------------
// Forward A.  Work item = (tile of kFwdTile samples, chunk of rows).  Each
// thread owns kFwdS samples and sums over the chunk's voxels row by row (rows
// pass through shared memory rows_staged at a time):
//   O(t) = sum_x c_x [a W + d (y.W) y] = Sa W + V,   W = beta G v,
// with the row structure used twice: y_y (diagonal G) is constant along a row,
// so V_y = y_y sum_row f; and rows far from every sample of the warp skip the
// near-FFP series test entirely.  Row sums are folded into the chunk sums with
// compensated additions.  The item writes p_k . O(t) to its partial slot.
template <typename R, typename CIN, bool DIAG, int MAXF>
__device__ __forceinline__ void forward_item(const PairBatch<R, MAXF> &B, int64_t item,
                                             unsigned char *smem_raw)
{
    const PairFrame<R> &F = B.f[find_frame(B, item)];
    const int64_t local = F.order ? F.order[item - F.item0] : item - F.item0;
    const int chunk = (int)(local / F.n_tiles);
    const int tile = (int)(local % F.n_tiles);
    const int nx = F.nx;
    const int j0 = chunk * F.chunk;
    const int nr = min(F.chunk, F.ny - j0);

    const int RB = F.rows_staged;
    R A1, D1;  // the closed form at u = near_u (what clamped pairs received)
    Lang<R>::ad_far(Lang<R>::near_u, A1, D1);
    // Shared memory: xcol [nx], then per staging copy yrow [RB] and RB rows
    // of (x_i, c_ji) pairs.
    const int lane_id = threadIdx.x & 31;
    V2<R> *s_x = reinterpret_cast<V2<R> *>(smem_raw);
    V2<R> *s_y = s_x + nx + (MPI_FWD_WSTAGE ? (threadIdx.x >> 5) * (RB + RB * nx) : 0);
    V2<R> *s_xc = s_y + RB;
    const CIN *cin = reinterpret_cast<const CIN *>(F.in);
    for (int k = threadIdx.x; k < nx; k += kFwdThreads) s_x[k] = F.xcol[k];
    if (MPI_FWD_WSTAGE) __syncthreads();  // xcol is read by every warp's staging

    R Rx[kFwdS], Ry[kFwdS], Wx[kFwdS], Wy[kFwdS];
    int64_t t[kFwdS];
#pragma unroll
    for (int s = 0; s < kFwdS; ++s) {
#if MPI_FWD_WARP_RUN
        // a warp's kFwdS x 32 samples are one consecutive run of the
        // trajectory (a compact extent: narrower closed-form column segments)
        t[s] = (int64_t)tile * kFwdTile + (threadIdx.x >> 5) * (32 * kFwdS) + s * 32 + (threadIdx.x & 31);
#else
        t[s] = (int64_t)tile * kFwdTile + s * kFwdThreads + threadIdx.x;
#endif
        const V4<R> q = F.rw[t[s] < F.T ? t[s] : F.T - 1];
        Rx[s] = q.x; Ry[s] = q.y; Wx[s] = q.z; Wy[s] = q.w;
    }
    R Sa[kFwdS], Vx[kFwdS], Vy[kFwdS], cSa[kFwdS], cVx[kFwdS], cVy[kFwdS];
#pragma unroll
    for (int s = 0; s < kFwdS; ++s) Sa[s] = Vx[s] = Vy[s] = cSa[s] = cVx[s] = cVy[s] = R(0);
    // Extent of the warp's samples (prescaled), for the far-field segments.
    R wx_lo = Rx[0], wx_hi = Rx[0], wy_lo = Ry[0], wy_hi = Ry[0];
#pragma unroll
    for (int s = 1; s < kFwdS; ++s) {
        wx_lo = min(wx_lo, Rx[s]); wx_hi = max(wx_hi, Rx[s]);
        wy_lo = min(wy_lo, Ry[s]); wy_hi = max(wy_hi, Ry[s]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        wx_lo = min(wx_lo, __shfl_xor_sync(0xffffffffu, wx_lo, o));
        wx_hi = max(wx_hi, __shfl_xor_sync(0xffffffffu, wx_hi, o));
        wy_lo = min(wy_lo, __shfl_xor_sync(0xffffffffu, wy_lo, o));
        wy_hi = max(wy_hi, __shfl_xor_sync(0xffffffffu, wy_hi, o));
    }
    constexpr R kUv = vfar_threshold<R, false>();
    // Column origin and inverse pitch of the prescaled grid (for the per-row
    // segment bounds below; read from global memory, the shared copy is not
    // yet visible here).
    const R x0c = F.xcol[0].x;
    const R inv_h = R(1) / (nx > 1 ? F.xcol[1].x - x0c : R(1));
    const R ax_lo = wx_lo - x0c, ax_hi = wx_hi - x0c;

    // Rows of the chunk are staged RB at a time.
#pragma unroll 1
    for (int jb = j0; jb < j0 + nr; jb += RB) {
        const int nrb = min(RB, j0 + nr - jb);
        if (MPI_FWD_WSTAGE) {
            __syncwarp();  // this warp's previous rows are consumed
            for (int k = lane_id; k < nrb * nx; k += 32)
                s_xc[k] = V2<R>{s_x[k % nx].x, R(cin[(int64_t)jb * nx + k])};
            for (int k = lane_id; k < nrb; k += 32) s_y[k] = F.yrow[jb + k];
            __syncwarp();
        } else {
            __syncthreads();
            for (int k = threadIdx.x; k < nrb * nx; k += kFwdThreads)
                s_xc[k] = V2<R>{s_x[k % nx].x, R(cin[(int64_t)jb * nx + k])};
            for (int k = threadIdx.x; k < nrb; k += kFwdThreads) s_y[k] = F.yrow[jb + k];
            __syncthreads();
        }

#pragma unroll 1
    for (int r = 0; r < nrb; ++r) {
        const V2<R> yr = s_y[r];
        const V2<R> *xcrow = s_xc + r * nx;
        R oy[kFwdS], ox[kFwdS], yy2[kFwdS], yyW[kFwdS];
        R sa[kFwdS], vx[kFwdS], fy[kFwdS];
        bool near = false;
#pragma unroll
        for (int s = 0; s < kFwdS; ++s) {
            oy[s] = yr.y - Ry[s];
            ox[s] = yr.x - Rx[s];
            yy2[s] = oy[s] * oy[s];
            yyW[s] = oy[s] * Wy[s];
            near |= yy2[s] < Lang<R>::near_u;
            sa[s] = vx[s] = fy[s] = R(0);
        }
        if (DIAG) {
            // Columns [lo, hi] may hold a pair of this warp with u < vfar_u
            // (widened by one column and a relative margin on each side);
            // outside them every pair takes the asymptotic form.
            int lo = 1, hi = 0;  // empty
            {
                const R gy = max(R(0), max(wy_lo - yr.y, yr.y - wy_hi));
                const R gy2 = gy * gy;
                if (gy2 < kUv) {
                    // sqrt(kUv - gy2) as x rsqrt(x) with an FP32 estimate (x >=
                    // ulp(kUv) > 0); its error and that of the inverse pitch are
                    // far inside the 1e-4 relative and one-column margins.
                    const R x = kUv - gy2;
                    const R w = x * R(rsqrt_approx(float(x))) * R(1.0001);
                    const R ia = (ax_lo - w) * inv_h, ib = (ax_hi + w) * inv_h;
                    const R fl = min(max(floor(min(ia, ib)) - R(1), R(0)), R(nx));
                    const R fh = min(max(ceil(max(ia, ib)) + R(1), R(-1)), R(nx - 1));
                    lo = (int)fl;
                    hi = (int)fh;
                }
            }
            if (lo > hi) {
                fwd_row_vfar<R>(0, nx, xcrow, Rx, yy2, Wx, yyW, sa, vx, fy);
            } else {
                fwd_row_vfar<R>(0, lo, xcrow, Rx, yy2, Wx, yyW, sa, vx, fy);
                if (!__any_sync(0xffffffffu, near)) {
                    // Every pair of this row has u >= yy2 >= near_u: closed form only.
                    fwd_row_far<R, false>(lo, hi + 1, xcrow, Rx, yy2, Wx, yyW, sa, vx, fy);
                } else {
                    // Closed form with u clamped to near_u, then the exact series
                    // for the few pairs of this thread that are really near
                    // (all inside [lo, hi]: u < near_u < vfar_u).
                    fwd_row_far<R, true>(lo, hi + 1, xcrow, Rx, yy2, Wx, yyW, sa, vx, fy);
#pragma unroll
                    for (int s = 0; s < kFwdS; ++s)
                        if (yy2[s] < Lang<R>::near_u)
                            fwd_near_fix<R>(nx, xcrow, Rx[s], yy2[s], Wx[s], yyW[s], A1, D1,
                                            F.near_cols, sa[s], vx[s], fy[s]);
                }
                fwd_row_vfar<R>(hi + 1, nx, xcrow, Rx, yy2, Wx, yyW, sa, vx, fy);
            }
#pragma unroll
            for (int s = 0; s < kFwdS; ++s) {
                kahan_add(Sa[s], cSa[s], sa[s]);
                kahan_add(Vx[s], cVx[s], vx[s]);
                kahan_add(Vy[s], cVy[s], oy[s] * fy[s]);
            }
        } else {
            // General case: near-FFP pairs possible (or a non-diagonal G).
#pragma unroll 2
            for (int i = 0; i < nx; ++i) {
                const V2<R> xi = s_x[i];
                const R ci = xcrow[i].y;
#pragma unroll
                for (int s = 0; s < kFwdS; ++s) {
                    const R yx = xi.x + ox[s];
                    const R yy = DIAG ? oy[s] : xi.y + oy[s];
                    const R u = fmx(yx, yx, yy * yy);
                    R a, d;
                    lang_checked<R, false>(u, a, d);
                    sa[s] = fmx(ci, a, sa[s]);
                    const R f = ci * d * fmx(yx, Wx[s], yy * Wy[s]);
                    vx[s] = fmx(f, yx, vx[s]);
                    fy[s] = fmx(f, yy, fy[s]);
                }
            }
#pragma unroll
            for (int s = 0; s < kFwdS; ++s) {
                kahan_add(Sa[s], cSa[s], sa[s]);
                kahan_add(Vx[s], cVx[s], vx[s]);
                kahan_add(Vy[s], cVy[s], fy[s]);
            }
        }
    }
    }

    R *part = reinterpret_cast<R *>(F.part);
#pragma unroll
    for (int s = 0; s < kFwdS; ++s) {
        if (t[s] < F.T) {
            const R Ox = Sa[s] * Wx[s] + Vx[s];
            const R Oy = Sa[s] * Wy[s] + Vy[s];
            for (int k = 0; k < F.n_ch; ++k)
                part[((int64_t)chunk * F.n_ch + k) * F.T + t[s]] = F.p[2 * k] * Ox + F.p[2 * k + 1] * Oy;
        }
    }
}

// ---------------------------------------------------------------------------
// One staged sample against this thread's kAdjV voxels of a column (adjoint /
// beta-derivative): blk[v] += f1 (u.W) + f2 y^T S y.  FAR: the warp's voxel
// box is provably outside the near-FFP range for this sample.
template <typename R, bool DBETA, int MODE>
__device__ __forceinline__ void lang_mode(R u, R &f1, R &f2)
{
    if constexpr (MODE == 2) lang_vfar<R, DBETA>(u, f1, f2);
    else if constexpr (MODE == 1) lang_far<R, DBETA>(u, f1, f2);
    else lang_checked<R, DBETA>(u, f1, f2);
}

// MODE 2: the warp's voxel box is provably in the asymptotic range for this
// sample; 1: in the closed-form range; 0: near pairs possible.
template <typename R, bool DIAG, bool DBETA, int MODE>
__device__ __forceinline__ void adj_sample(const V2<R> rr, const V4<R> q, const V2<R> xc,
                                           const R (&yrow_x)[kAdjV], const R (&yrow_y)[kAdjV],
                                           R (&blk)[kAdjV])
{
    if (DIAG) {
        const R yx = xc.x - rr.x;
        const R yx2 = yx * yx;
        const R Q0 = q.y * yx2, Q1 = q.z * yx;
#pragma unroll
        for (int v = 0; v < kAdjV; ++v) {
            const R yy = yrow_y[v] - rr.y;
            const R u = fmx(yy, yy, yx2);
            const R P = fmx(yy, fmx(q.w, yy, Q1), Q0);
            if constexpr (MODE == 2) {
                blk[v] = pair_acc_vfar<R, DBETA>(u, q.x, P, blk[v]);
            } else {
                R f1, f2;
                lang_mode<R, DBETA, MODE>(u, f1, f2);
                blk[v] += fmx(f1, q.x, f2 * P);
            }
        }
    } else {
        const R ox = xc.x - rr.x, oy = xc.y - rr.y;
#pragma unroll
        for (int v = 0; v < kAdjV; ++v) {
            const R yx = ox + yrow_x[v];
            const R yy = oy + yrow_y[v];
            const R u = fmx(yx, yx, yy * yy);
            const R quad = fmx(yx, fmx(q.y, yx, q.z * yy), q.w * yy * yy);
            if constexpr (MODE == 2) {
                blk[v] = pair_acc_vfar<R, DBETA>(u, q.x, quad, blk[v]);
            } else {
                R f1, f2;
                lang_mode<R, DBETA, MODE>(u, f1, f2);
                blk[v] += fmx(f1, q.x, f2 * quad);
            }
        }
    }
}

#ifdef __CUDACC__
// Two staged samples (2h, 2h + 1) against this thread's kAdjV voxels in the
// asymptotic range, diagonal G, packed: a = (-x_e, -x_o, -y_e, -y_o) of B r,
// b = (uW_e, uW_o, Sxx_e, Sxx_o), c = (S2xy_e, S2xy_o, Syy_e, Syy_o); xc2 =
// (x_c, x_c) of the thread's column, yr2[v] = (y_v, y_v).  Lane-wise the
// same operations, in the same order, as adj_sample's MODE 2 on each sample.
template <bool DBETA>
__device__ __forceinline__ void adj_pair2_vfar_diag(const float4 a, const float4 b, const float4 c,
                                                    const float2 xc2, const float2 (&yr2)[kAdjV],
                                                    float2 (&blk2)[kAdjV])
{
    const float2 nry = make_float2(a.z, a.w);
    const float2 uW = make_float2(b.x, b.y), Sxx = make_float2(b.z, b.w);
    const float2 S2xy = make_float2(c.x, c.y), Syy = make_float2(c.z, c.w);
    const float2 yx = __fadd2_rn(xc2, make_float2(a.x, a.y));
    const float2 yx2 = __fmul2_rn(yx, yx);
    const float2 Q0 = __fmul2_rn(Sxx, yx2), Q1 = __fmul2_rn(S2xy, yx);
    const float2 nuW = __fmul2_rn(uW, make_float2(-1.0f, -1.0f));
#pragma unroll
    for (int v = 0; v < kAdjV; ++v) {
        const float2 yy = __fadd2_rn(yr2[v], nry);
        const float2 u = __ffma2_rn(yy, yy, yx2);
        const float2 P = __ffma2_rn(yy, __ffma2_rn(Syy, yy, Q1), Q0);
        const float2 iz = make_float2(Lang<float>::iz_vfar(u.x), Lang<float>::iz_vfar(u.y));
        if constexpr (DBETA) {
            const float2 iz2 = __fmul2_rn(iz, iz);
            const float2 t = __ffma2_rn(__fmul2_rn(iz2, P), make_float2(-2.0f, -2.0f), uW);
            blk2[v] = __ffma2_rn(iz2, t, blk2[v]);
        } else {
            const float2 t = __fmul2_rn(P, __ffma2_rn(iz, make_float2(2.0f, 2.0f), make_float2(-1.0f, -1.0f)));
            const float2 w = __ffma2_rn(iz, t, nuW);
            blk2[v] = __ffma2_rn(iz, __ffma2_rn(iz, w, uW), blk2[v]);
        }
    }
}
#endif

// ---------------------------------------------------------------------------
// Adjoint A^T (DBETA = false) and the beta-derivative (DBETA = true).
// Work item = (tile of 32 x kAdjTileY voxels, chunk of samples).  Lane =
// column; each thread owns kAdjV consecutive rows of its column, each warp a
// 32 x kAdjV box.  Samples are staged in shared memory (kAdjStageCopies
// copies), kAdjBlock at a time, as
//   (B r_t) and (u.W, W_x u_x, W_x u_y + W_y u_x, W_y u_y),  u = sum_k s_k p_k,
// so that the pair term u^T J w = a (u.W) + d (y.W)(y.u) is
//   f1 uW + f2 (yx^2 Sxx + yx yy S2xy + yy^2 Syy)
// with (f1, f2) = (a, d) for A^T and (L', L''/z) for d/dbeta.  Per warp and
// staged block a ballot marks the samples whose distance to the warp's voxel
// box keeps every pair in the closed-form range.  ONEBLK: every chunk is at
// most one staged block (the chunk sum is that block's sum: no compensation
// needed, the same result as the compensated sum).
template <typename R, bool DIAG, bool DBETA, int MAXF, bool ONEBLK>
__device__ __forceinline__ void adjoint_item(const PairBatch<R, MAXF> &B, int64_t item)
{
    // PACK: the FP32 diagonal-G asymptotic tier runs packed (kAdjPack), from
    // a second copy of the staged samples in pairs (three float4 per pair).
    constexpr bool PACK = kAdjPack && sizeof(R) == 4 && DIAG;
    __shared__ V2<R> s_rw[kAdjStageCopies][kAdjBlock];
    __shared__ V4<R> s_qw[kAdjStageCopies][kAdjBlock];
    __shared__ float4 s_pkw[PACK ? kAdjStageCopies : 1][PACK ? 3 * kAdjBlock / 2 : 1];
    __shared__ uint32_t s_far[kAdjWarps][kAdjBlock / 32];
    __shared__ uint32_t s_vfar[kAdjWarps][kAdjBlock / 32];
    __shared__ double s_red[kAdjThreads / 32];

    const PairFrame<R> &F = B.f[find_frame(B, item)];
    const int64_t local = F.order ? F.order[item - F.item0] : item - F.item0;
    const int chunk = (int)(local / F.n_tiles);
    const int tile = (int)(local % F.n_tiles);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#if MPI_ADJ_BOX16
    // warp box 16 columns x 16 rows (lanes 0-15 and 16-31 take two
    // kAdjV-row bands of the same 16 columns; the block's 4 warps 2 x 2)
    static_assert(kAdjWarps == 4 && kAdjV == 8, "16 x 16 warp boxes need 4 warps of 8-row threads");
    const int i = (tile % F.tiles_x) * kAdjTileX + (warp & 1) * 16 + (lane & 15);
    const int jb = (tile / F.tiles_x) * kAdjTileY + (warp >> 1) * 16 + (lane >> 4) * kAdjV;
#else
    const int i = (tile % F.tiles_x) * kAdjTileX + lane;
    const int jb = (tile / F.tiles_x) * kAdjTileY + warp * kAdjV;
#endif
    V2<R> *s_r = s_rw[MPI_ADJ_WSTAGE ? warp : 0];
    V4<R> *s_q = s_qw[MPI_ADJ_WSTAGE ? warp : 0];
    float4 *s_pk = s_pkw[PACK && MPI_ADJ_WSTAGE ? warp : 0];
    // stager: this warp's lanes (one copy per warp) or the block's threads
    const int st_id = MPI_ADJ_WSTAGE ? lane : (int)threadIdx.x;
    constexpr int st_n = MPI_ADJ_WSTAGE ? 32 : kAdjThreads;
    const int ic = min(i, F.nx - 1);

    const V2<R> xc = F.xcol[ic];
    R yrow_y[kAdjV], yrow_x[kAdjV];
#pragma unroll
    for (int v = 0; v < kAdjV; ++v) {
        const V2<R> q = F.yrow[min(jb + v, F.ny - 1)];
        yrow_x[v] = q.x;
        yrow_y[v] = q.y;
    }
    const float2 xc2 = make_float2(float(xc.x), float(xc.x));
    float2 yr2[PACK ? kAdjV : 1];
#pragma unroll
    for (int v = 0; v < (PACK ? kAdjV : 1); ++v) yr2[v] = make_float2(float(yrow_y[v]), float(yrow_y[v]));
    // Voxel box of this warp in prescaled coordinates (conservative).
    R bx_lo = xc.x, bx_hi = xc.x, by_lo = xc.y, by_hi = xc.y;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        bx_lo = min(bx_lo, __shfl_xor_sync(0xffffffffu, bx_lo, o));
        bx_hi = max(bx_hi, __shfl_xor_sync(0xffffffffu, bx_hi, o));
        by_lo = min(by_lo, __shfl_xor_sync(0xffffffffu, by_lo, o));
        by_hi = max(by_hi, __shfl_xor_sync(0xffffffffu, by_hi, o));
    }
    {
        R ry_lo = yrow_y[0], ry_hi = yrow_y[0], rx_lo = yrow_x[0], rx_hi = yrow_x[0];
#pragma unroll
        for (int v = 1; v < kAdjV; ++v) {
            ry_lo = min(ry_lo, yrow_y[v]); ry_hi = max(ry_hi, yrow_y[v]);
            rx_lo = min(rx_lo, yrow_x[v]); rx_hi = max(rx_hi, yrow_x[v]);
        }
#if MPI_ADJ_BOX16
        // the two halves of the warp hold different rows: the box spans both
        ry_lo = min(ry_lo, __shfl_xor_sync(0xffffffffu, ry_lo, 16));
        ry_hi = max(ry_hi, __shfl_xor_sync(0xffffffffu, ry_hi, 16));
        rx_lo = min(rx_lo, __shfl_xor_sync(0xffffffffu, rx_lo, 16));
        rx_hi = max(rx_hi, __shfl_xor_sync(0xffffffffu, rx_hi, 16));
#endif
        bx_lo += rx_lo; bx_hi += rx_hi; by_lo += ry_lo; by_hi += ry_hi;
    }

    const int64_t t0 = (int64_t)chunk * F.chunk;
    const int64_t t1 = min(F.T, t0 + F.chunk);
    const R *sin = reinterpret_cast<const R *>(DBETA ? F.in2 : F.in);

    R acc[kAdjV], comp[kAdjV];
#pragma unroll
    for (int v = 0; v < kAdjV; ++v) acc[v] = comp[v] = R(0);

#pragma unroll 1
    for (int64_t tb = t0; tb < t1; tb += kAdjBlock) {
        const int nb = (int)min((int64_t)kAdjBlock, t1 - tb);
        // the previous block of staged samples is consumed
        if (MPI_ADJ_WSTAGE) __syncwarp();
        else __syncthreads();
        for (int k = st_id; k < nb; k += st_n) {
            const int64_t t = tb + k;
            const V4<R> q = F.rw[t];
            R ux = R(0), uy = R(0);
            for (int c = 0; c < F.n_ch; ++c) {
                const R sv = sin[(int64_t)c * F.T + t];
                ux += sv * F.p[2 * c];
                uy += sv * F.p[2 * c + 1];
            }
            const V4<R> sq = V4<R>{ux * q.z + uy * q.w, q.z * ux, q.z * uy + q.w * ux, q.w * uy};
            s_r[k] = V2<R>{q.x, q.y};
            s_q[k] = sq;
            if constexpr (PACK) {
                float *pb = reinterpret_cast<float *>(s_pk + 3 * (k >> 1)) + (k & 1);
                pb[0] = -float(q.x);
                pb[2] = -float(q.y);
                pb[4] = float(sq.x);
                pb[6] = float(sq.y);
                pb[8] = float(sq.z);
                pb[10] = float(sq.w);
            }
        }
        if (MPI_ADJ_WSTAGE) __syncwarp();
        else __syncthreads();
        // Far / very-far flags of this warp for the staged samples.
        for (int m = 0; m < kAdjBlock / 32; ++m) {
            const int k = m * 32 + lane;
            bool far = true, vfar = true;
            if (k < nb) {
                const V2<R> q = s_r[k];
                const R ddx = max(R(0), max(bx_lo - q.x, q.x - bx_hi));
                const R ddy = max(R(0), max(by_lo - q.y, q.y - by_hi));
                const R d2 = fmx(ddy, ddy, ddx * ddx);
                far = d2 >= Lang<R>::near_u;
                vfar = d2 >= vfar_threshold<R, DBETA>();
            }
            const uint32_t bits = __ballot_sync(0xffffffffu, far);
            const uint32_t vbits = __ballot_sync(0xffffffffu, vfar);
            if (lane == 0) {
                s_far[warp][m] = bits;
                s_vfar[warp][m] = vbits;
            }
        }
        __syncwarp();

        R blk[kAdjV];
#pragma unroll
        for (int v = 0; v < kAdjV; ++v) blk[v] = R(0);
        // 32 staged samples share one word of far flags: runs of 32 far
        // samples take a loop without per-sample tests.
#pragma unroll 1
        for (int k0 = 0; k0 < nb; k0 += 32) {
            const uint32_t mask = s_far[warp][k0 >> 5];
            const uint32_t vmask = s_vfar[warp][k0 >> 5];
            const int kn = min(32, nb - k0);
            if (kn == 32 && vmask == 0xffffffffu) {
                if constexpr (PACK) {
                    // the group's even and odd samples in the two lanes, then
                    // added into the block sums
                    float2 blk2[kAdjV];
#pragma unroll
                    for (int v = 0; v < kAdjV; ++v) blk2[v] = make_float2(0.0f, 0.0f);
#pragma unroll kAdjUnrollVfar
                    for (int h = k0 >> 1; h < (k0 >> 1) + 16; ++h)
                        adj_pair2_vfar_diag<DBETA>(s_pk[3 * h], s_pk[3 * h + 1], s_pk[3 * h + 2], xc2, yr2, blk2);
#pragma unroll
                    for (int v = 0; v < kAdjV; ++v) blk[v] += blk2[v].x + blk2[v].y;
                } else {
#pragma unroll kAdjUnrollVfar
                    for (int k = k0; k < k0 + 32; ++k)
                        adj_sample<R, DIAG, DBETA, 2>(s_r[k], s_q[k], xc, yrow_x, yrow_y, blk);
                }
            } else if (kn == 32 && mask == 0xffffffffu) {
#pragma unroll 2
                for (int k = k0; k < k0 + 32; ++k)
                    adj_sample<R, DIAG, DBETA, 1>(s_r[k], s_q[k], xc, yrow_x, yrow_y, blk);
            } else {
#pragma unroll 1
                for (int k = k0; k < k0 + kn; ++k) {
                    if ((vmask >> (k - k0)) & 1u)
                        adj_sample<R, DIAG, DBETA, 2>(s_r[k], s_q[k], xc, yrow_x, yrow_y, blk);
                    else if ((mask >> (k - k0)) & 1u)
                        adj_sample<R, DIAG, DBETA, 1>(s_r[k], s_q[k], xc, yrow_x, yrow_y, blk);
                    else
                        adj_sample<R, DIAG, DBETA, 0>(s_r[k], s_q[k], xc, yrow_x, yrow_y, blk);
                }
            }
        }
#pragma unroll
        for (int v = 0; v < kAdjV; ++v) {
            if (ONEBLK) acc[v] += blk[v];
            else kahan_add(acc[v], comp[v], blk[v]);
        }
    }

    if constexpr (!DBETA) {
        R *part = reinterpret_cast<R *>(F.part);
        const int64_t N = (int64_t)F.nx * F.ny;
        if (i < F.nx) {
#pragma unroll
            for (int v = 0; v < kAdjV; ++v)
                if (jb + v < F.ny) part[(int64_t)chunk * N + (int64_t)(jb + v) * F.nx + i] = acc[v];
        }
    } else {
        const R *c = reinterpret_cast<const R *>(F.in);
        double sum = 0.0;
        if (i < F.nx) {
#pragma unroll
            for (int v = 0; v < kAdjV; ++v)
                if (jb + v < F.ny) sum += double(c[(int64_t)(jb + v) * F.nx + i]) * double(acc[v]);
        }
        sum = block_sum<double, kAdjThreads>(sum, s_red);
        if (threadIdx.x == 0) reinterpret_cast<double *>(F.part)[local] = sum;
    }
}

// ---------------------------------------------------------------------------
// Launch forms.  One block per work item (the hardware block scheduler hands
// out items), or persistent: gridDim.x resident blocks pull item indices from
// a device counter until the items run out; the last block to leave resets
// the counter for the next launch (no block ever waits for another).  Both
// give identical results: an item's arithmetic does not depend on which block
// runs it.

__device__ __forceinline__ bool queue_next(unsigned long long *queue, int64_t n_items,
                                           long long *s_item, int64_t &item)
{
    if (threadIdx.x == 0) *s_item = (long long)atomicAdd(&queue[0], 1ull);
    __syncthreads();
    item = *s_item;
    __syncthreads();
    return item < n_items;
}

__device__ __forceinline__ void queue_leave(unsigned long long *queue)
{
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(&queue[1], 1ull) == gridDim.x - 1) {
            queue[0] = 0;
            queue[1] = 0;
            __threadfence();
        }
    }
}

// DM selects the pair-math branch: 0 = general G, 1 = diagonal G, 2 = per
// frame (mixed batches; the frame's `diag` flag picks, uniformly per block).
template <typename R, typename CIN, int DM, int MAXF>
__device__ __forceinline__ void forward_dispatch(const PairBatch<R, MAXF> &B, int64_t item,
                                                 unsigned char *smem_raw)
{
    if constexpr (DM == 2) {
        if (B.f[find_frame(B, item)].diag) forward_item<R, CIN, true, MAXF>(B, item, smem_raw);
        else forward_item<R, CIN, false, MAXF>(B, item, smem_raw);
    } else {
        forward_item<R, CIN, DM == 1, MAXF>(B, item, smem_raw);
    }
}

template <typename R, int DM, bool DBETA, int MAXF, bool ONEBLK>
__device__ __forceinline__ void adjoint_dispatch(const PairBatch<R, MAXF> &B, int64_t item)
{
    if constexpr (DM == 2) {
        if (B.f[find_frame(B, item)].diag) adjoint_item<R, true, DBETA, MAXF, ONEBLK>(B, item);
        else adjoint_item<R, false, DBETA, MAXF, ONEBLK>(B, item);
    } else {
        adjoint_item<R, DM == 1, DBETA, MAXF, ONEBLK>(B, item);
    }
}

template <typename R, typename CIN, int DM, int MAXF>
__global__ void __launch_bounds__(kFwdThreads, sizeof(R) == 4 ? MPI_FWD_MINB : 2)
k_forward(const __grid_constant__ PairBatch<R, MAXF> B)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    forward_dispatch<R, CIN, DM, MAXF>(B, blockIdx.x, smem_raw);
}

template <typename R, typename CIN, int DM, int MAXF>
__global__ void __launch_bounds__(kFwdThreads, sizeof(R) == 4 ? MPI_FWD_MINB : 2)
k_forward_persistent(const __grid_constant__ PairBatch<R, MAXF> B, int64_t n_items,
                     unsigned long long *queue)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ long long s_item;
    int64_t item;
    while (queue_next(queue, n_items, &s_item, item)) {
        forward_dispatch<R, CIN, DM, MAXF>(B, item, smem_raw);
        __syncthreads();
    }
    queue_leave(queue);
}

template <typename R, int DM, bool DBETA, int MAXF, bool ONEBLK = false>
__global__ void __launch_bounds__(kAdjThreads, sizeof(R) == 4 ? MPI_ADJ_MINB : 8 / MPI_ADJ_WARPS)
k_adjoint(const __grid_constant__ PairBatch<R, MAXF> B)
{
    adjoint_dispatch<R, DM, DBETA, MAXF, ONEBLK>(B, blockIdx.x);
}

template <typename R, int DM, bool DBETA, int MAXF, bool ONEBLK = false>
__global__ void __launch_bounds__(kAdjThreads, sizeof(R) == 4 ? MPI_ADJ_MINB : 8 / MPI_ADJ_WARPS)
k_adjoint_persistent(const __grid_constant__ PairBatch<R, MAXF> B, int64_t n_items,
                     unsigned long long *queue)
{
    __shared__ long long s_item;
    int64_t item;
    while (queue_next(queue, n_items, &s_item, item)) {
        adjoint_dispatch<R, DM, DBETA, MAXF, ONEBLK>(B, item);
        __syncthreads();
    }
    queue_leave(queue);
}

#endif  // __CUDACC__

}  // namespace mpi
