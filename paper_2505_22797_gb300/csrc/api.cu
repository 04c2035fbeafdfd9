// C ABI entry points: argument validation, scratch sizing and dispatch of the
// operator calls (forward A, adjoint A^T, d/dbeta).
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstring>
#include <mutex>
#include <vector>

#include "graph.cuh"
#include "pair_ops.cuh"

namespace mpi {

static thread_local char g_err[512] = "";

void set_error(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}
const char *last_error() { return g_err; }

int Scratch::allocate()
{
    if (total_ == 0) return MPI_OK;
    if (const char *f = getenv("MPI_FAULT")) {
        if (strcmp(f, "alloc") == 0) {
            set_error("scratch allocation of %zu bytes failed (injected by MPI_FAULT=alloc)", total_);
            return MPI_ERR_NOMEM;
        }
    }
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&base_), total_, stream_);
    if (e != cudaSuccess) {
        base_ = nullptr;
        set_error("cudaMallocAsync(%zu) failed: %s", total_, cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? MPI_ERR_NOMEM : MPI_ERR_CUDA;
    }
    return MPI_OK;
}

void Scratch::release()
{
    if (base_) cudaFreeAsync(base_, stream_);
    base_ = nullptr;
}

// ---------------------------------------------------------------------------
// Launch counter and optional event timing of the operator kernels.

static std::atomic<long long> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void note_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

namespace {
struct ProfRecord {
    int cls;
    cudaEvent_t ev[2];
};
std::mutex g_prof_mu;
bool g_prof_on = false;
std::vector<ProfRecord> g_prof_pending;
std::vector<cudaEvent_t> g_prof_free;
long long g_prof_n[kProfClasses] = {0, 0, 0, 0};
double g_prof_ms[kProfClasses] = {0, 0, 0, 0};

cudaEvent_t take_event()
{
    if (!g_prof_free.empty()) {
        cudaEvent_t e = g_prof_free.back();
        g_prof_free.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Resolve recorded event pairs into per-class totals (caller holds the lock).
int drain_pending()
{
    for (const ProfRecord &r : g_prof_pending) {
        float ms = 0.f;
        if (cudaEventSynchronize(r.ev[1]) != cudaSuccess ||
            cudaEventElapsedTime(&ms, r.ev[0], r.ev[1]) != cudaSuccess) {
            set_error("profiling event query failed");
            return MPI_ERR_CUDA;
        }
        g_prof_n[r.cls] += 1;
        g_prof_ms[r.cls] += ms;
        g_prof_free.push_back(r.ev[0]);
        g_prof_free.push_back(r.ev[1]);
    }
    g_prof_pending.clear();
    return MPI_OK;
}
}  // namespace

ProfScope::ProfScope(int cls, cudaStream_t st) : cls_(cls), st_(st), on_(false)
{
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (!g_prof_on) return;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st_, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
    ev_[0] = take_event();
    ev_[1] = take_event();
    if (ev_[0] && ev_[1] && cudaEventRecord(ev_[0], st_) == cudaSuccess) on_ = true;
}

ProfScope::~ProfScope()
{
    if (!on_) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (cudaEventRecord(ev_[1], st_) == cudaSuccess) g_prof_pending.push_back({cls_, {ev_[0], ev_[1]}});
}

bool profile_enabled()
{
    std::lock_guard<std::mutex> lk(g_prof_mu);
    return g_prof_on;
}

CapturedGraph::~CapturedGraph()
{
    if (exec_) cudaGraphExecDestroy(exec_);  // freed once a replay in flight completes
    if (graph_) cudaGraphDestroy(graph_);
    if (cap_) cudaStreamDestroy(cap_);
}

int CapturedGraph::fail()
{
    if (exec_) cudaGraphExecDestroy(exec_);
    if (graph_) cudaGraphDestroy(graph_);
    exec_ = nullptr;
    graph_ = nullptr;
    (void)cudaGetLastError();  // a refused capture leaves no error for the direct path
    return MPI_ERR_UNSUPPORTED;
}

int CapturedGraph::launch(cudaStream_t st)
{
    MPI_TRY_CUDA(cudaGraphLaunch(exec_, st));
    note_launches((long long)nodes_);
    return MPI_OK;
}

long long CapturedGraph::counted_launches() { return mpi_kernel_launches(); }
void CapturedGraph::uncount_launches(long long n) { note_launches(-n); }

int device_sm_count()
{
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 132;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 132;
    return n > 0 ? n : 132;
}

// ---------------------------------------------------------------------------
// Validation.

int check_model(const mpi_model *m)
{
    if (!m) { set_error("model is NULL"); return MPI_ERR_INVALID; }
    if (!(m->beta > 0.0) || !std::isfinite(m->beta)) {
        set_error("beta must be positive and finite (got %g)", m->beta);
        return MPI_ERR_INVALID;
    }
    for (int k = 0; k < 4; ++k)
        if (!std::isfinite(m->G[k])) { set_error("G has a non-finite entry"); return MPI_ERR_INVALID; }
    const double det = m->G[0] * m->G[3] - m->G[1] * m->G[2];
    if (det == 0.0) { set_error("G is singular"); return MPI_ERR_INVALID; }
    if (m->n_ch != 1 && m->n_ch != 2) {
        set_error("n_ch must be 1 or 2 (got %d)", m->n_ch);
        return MPI_ERR_INVALID;
    }
    for (int k = 0; k < 2 * m->n_ch; ++k)
        if (!std::isfinite(m->p[k])) { set_error("p has a non-finite entry"); return MPI_ERR_INVALID; }
    return MPI_OK;
}

int check_grid(const mpi_grid_desc *g)
{
    if (!g) { set_error("grid is NULL"); return MPI_ERR_INVALID; }
    if (g->nx < 1 || g->ny < 1) {
        set_error("grid must have nx, ny >= 1 (got %d x %d)", g->nx, g->ny);
        return MPI_ERR_INVALID;
    }
    if ((int64_t)g->nx * g->ny > (int64_t)1 << 28) {
        set_error("grid of %d x %d voxels is larger than supported (2^28)", g->nx, g->ny);
        return MPI_ERR_UNSUPPORTED;
    }
    if (!(g->dx != 0.0) || !(g->dy != 0.0) || !std::isfinite(g->dx) || !std::isfinite(g->dy) ||
        !std::isfinite(g->x0) || !std::isfinite(g->y0)) {
        set_error("grid spacing must be nonzero and finite");
        return MPI_ERR_INVALID;
    }
    return MPI_OK;
}

int check_traj(const mpi_traj *t)
{
    if (!t) { set_error("trajectory is NULL"); return MPI_ERR_INVALID; }
    if (t->T < 0) { set_error("T must be >= 0 (got %lld)", (long long)t->T); return MPI_ERR_INVALID; }
    if (t->T > ((int64_t)1 << 34)) { set_error("T too large"); return MPI_ERR_UNSUPPORTED; }
    if (t->T > 0 && (!t->r || !t->v)) { set_error("trajectory arrays are NULL"); return MPI_ERR_INVALID; }
    return MPI_OK;
}

int check_dtype(mpi_dtype d)
{
    if (d != MPI_F32 && d != MPI_F64) { set_error("dtype must be MPI_F32 or MPI_F64"); return MPI_ERR_INVALID; }
    return MPI_OK;
}

ModelH to_host(const mpi_model *m)
{
    ModelH h;
    h.beta = m->beta;
    for (int k = 0; k < 4; ++k) h.G[k] = m->G[k];
    h.n_ch = m->n_ch;
    for (int k = 0; k < 4; ++k) h.p[k] = k < 2 * m->n_ch ? m->p[k] : 0.0;
    return h;
}
GridH to_host(const mpi_grid_desc *g) { return GridH{g->nx, g->ny, g->x0, g->y0, g->dx, g->dy}; }

// ---------------------------------------------------------------------------

template <typename R>
static int forward_impl(const ModelH &m, const GridH &g, const mpi_traj *tr, const void *c, void *s,
                        cudaStream_t st)
{
    const int64_t T = tr->T;
    if (T == 0) return MPI_OK;
    FwdSplit sp = forward_split(T, g.nx, g.ny, sizeof(R), forward_target_items());
    Scratch scr(st);
    const size_t o_geo = scr.reserve(geometry_bytes<R>(T, g.nx, g.ny));
    const size_t o_part = scr.reserve(forward_partial_bytes<R>(sp, m.n_ch, T));
    const size_t o_ord = scr.reserve(item_order_bytes<R>(&sp, nullptr));
    MPI_TRY(scr.allocate());
    const Geometry<R> geo = geometry_carve<R>(scr.at<char>(o_geo), T, g.nx, g.ny);
    MPI_TRY(prepare_geometry<R>(m, g, T, tr->r, tr->v, geo, st));
    MPI_TRY(prepare_item_orders<R>(g, T, geo, &sp, nullptr, scr.at<char>(o_ord), st));
    return launch_forward<R, R, R>(m, g, T, geo, sp, static_cast<const R *>(c), scr.at<R>(o_part),
                                   static_cast<R *>(s), st);
}

template <typename R>
static int adjoint_impl(const ModelH &m, const GridH &g, const mpi_traj *tr, const void *s, void *c,
                        cudaStream_t st)
{
    const int64_t T = tr->T;
    AdjSplit sp = adjoint_split(T, g.nx, g.ny, default_target_items(), sizeof(R));
    Scratch scr(st);
    const size_t o_geo = scr.reserve(geometry_bytes<R>(T, g.nx, g.ny));
    const size_t o_part = scr.reserve(adjoint_partial_bytes<R>(sp, g.nx, g.ny));
    const size_t o_ord = scr.reserve(item_order_bytes<R>(nullptr, &sp));
    MPI_TRY(scr.allocate());
    const Geometry<R> geo = geometry_carve<R>(scr.at<char>(o_geo), T, g.nx, g.ny);
    MPI_TRY(prepare_geometry<R>(m, g, T, tr->r, tr->v, geo, st));
    MPI_TRY(prepare_item_orders<R>(g, T, geo, nullptr, &sp, scr.at<char>(o_ord), st));
    return launch_adjoint<R, R>(m, g, T, geo, sp, static_cast<const R *>(s), scr.at<R>(o_part),
                                static_cast<R *>(c), nullptr, nullptr, nullptr, st);
}

template <typename R>
static int dbeta_impl(const ModelH &m, const GridH &g, const mpi_traj *tr, const void *c,
                      const void *gs, double *out, cudaStream_t st)
{
    const int64_t T = tr->T;
    AdjSplit sp = adjoint_split(T, g.nx, g.ny, default_target_items(), sizeof(R));
    Scratch scr(st);
    const size_t o_geo = scr.reserve(geometry_bytes<R>(T, g.nx, g.ny));
    const size_t o_part = scr.reserve(dbeta_partial_bytes(sp));
    const size_t o_ord = scr.reserve(item_order_bytes<R>(nullptr, &sp));
    MPI_TRY(scr.allocate());
    const Geometry<R> geo = geometry_carve<R>(scr.at<char>(o_geo), T, g.nx, g.ny);
    MPI_TRY(prepare_geometry<R>(m, g, T, tr->r, tr->v, geo, st));
    MPI_TRY(prepare_item_orders<R>(g, T, geo, nullptr, &sp, scr.at<char>(o_ord), st));
    return launch_dbeta<R>(m, g, T, geo, sp, static_cast<const R *>(c), static_cast<const R *>(gs),
                           scr.at<double>(o_part), out, st);
}

}  // namespace mpi

using namespace mpi;

extern "C" {

int mpi_forward(const mpi_model *model, const mpi_grid_desc *grid, const mpi_traj *traj,
                mpi_dtype dtype, const void *c, void *s, void *stream)
{
    MPI_TRY(check_model(model));
    MPI_TRY(check_grid(grid));
    MPI_TRY(check_traj(traj));
    MPI_TRY(check_dtype(dtype));
    if (traj->T > 0 && (!c || !s)) { set_error("c or s is NULL"); return MPI_ERR_INVALID; }
    const ModelH m = to_host(model);
    const GridH g = to_host(grid);
    return dtype == MPI_F32 ? forward_impl<float>(m, g, traj, c, s, as_stream(stream))
                            : forward_impl<double>(m, g, traj, c, s, as_stream(stream));
}

int mpi_adjoint(const mpi_model *model, const mpi_grid_desc *grid, const mpi_traj *traj,
                mpi_dtype dtype, const void *s, void *c_out, void *stream)
{
    MPI_TRY(check_model(model));
    MPI_TRY(check_grid(grid));
    MPI_TRY(check_traj(traj));
    MPI_TRY(check_dtype(dtype));
    if (!c_out || (traj->T > 0 && !s)) { set_error("s or c_out is NULL"); return MPI_ERR_INVALID; }
    const ModelH m = to_host(model);
    const GridH g = to_host(grid);
    return dtype == MPI_F32 ? adjoint_impl<float>(m, g, traj, s, c_out, as_stream(stream))
                            : adjoint_impl<double>(m, g, traj, s, c_out, as_stream(stream));
}

int mpi_dbeta(const mpi_model *model, const mpi_grid_desc *grid, const mpi_traj *traj,
              mpi_dtype dtype, const void *c, const void *g, double *dbeta_dev, void *stream)
{
    MPI_TRY(check_model(model));
    MPI_TRY(check_grid(grid));
    MPI_TRY(check_traj(traj));
    MPI_TRY(check_dtype(dtype));
    if (!dbeta_dev || (traj->T > 0 && (!c || !g))) {
        set_error("c, g or dbeta_dev is NULL");
        return MPI_ERR_INVALID;
    }
    const ModelH m = to_host(model);
    const GridH gh = to_host(grid);
    return dtype == MPI_F32 ? dbeta_impl<float>(m, gh, traj, c, g, dbeta_dev, as_stream(stream))
                            : dbeta_impl<double>(m, gh, traj, c, g, dbeta_dev, as_stream(stream));
}

const char *mpi_status_string(int status)
{
    switch (status) {
    case MPI_OK: return "ok";
    case MPI_ERR_INVALID: return "invalid argument";
    case MPI_ERR_CUDA: return "CUDA error";
    case MPI_ERR_NOMEM: return "out of device memory";
    case MPI_ERR_CALLBACK: return "denoiser callback failed";
    case MPI_ERR_TIMEOUT: return "device-side wait timed out";
    case MPI_ERR_UNSUPPORTED: return "unsupported";
    default: return "unknown status";
    }
}

const char *mpi_last_error_message(void) { return last_error(); }

long long mpi_kernel_launches(void) { return g_launches.load(); }

int mpi_profile_enable(int enable)
{
    std::lock_guard<std::mutex> lk(g_prof_mu);
    const int st = drain_pending();
    for (int c = 0; c < kProfClasses; ++c) {
        g_prof_n[c] = 0;
        g_prof_ms[c] = 0.0;
    }
    g_prof_on = enable != 0;
    return st;
}

int mpi_profile_read(int kernel_class, long long *launches, double *total_ms)
{
    if (kernel_class < 0 || kernel_class >= kProfClasses || !launches || !total_ms) {
        set_error("invalid profile query");
        return MPI_ERR_INVALID;
    }
    std::lock_guard<std::mutex> lk(g_prof_mu);
    MPI_TRY(drain_pending());
    *launches = g_prof_n[kernel_class];
    *total_ms = g_prof_ms[kernel_class];
    return MPI_OK;
}

int mpi_version(void) { return 100; }

}  // extern "C"
