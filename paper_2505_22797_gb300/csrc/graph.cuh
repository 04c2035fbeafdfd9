// CUDA-graph capture of launch runs for the library's solve drivers (host
// code).
#pragma once

#include "common.cuh"

namespace mpi {

// True while mpi_profile_enable(1) is in effect (per-launch event timing).
bool profile_enabled();

// A run of launches captured once as a CUDA graph and replayed.  The
// capture uses a private stream in thread-local capture mode (the caller's
// stream may be the legacy default stream, which cannot be captured); the
// replays go to the caller's stream.  Launches made while capturing are not
// counted by mpi_kernel_launches(); each replay counts the graph's nodes.
class CapturedGraph {
  public:
    CapturedGraph() = default;
    ~CapturedGraph();
    CapturedGraph(const CapturedGraph &) = delete;
    CapturedGraph &operator=(const CapturedGraph &) = delete;
    // Captures what enqueue(stream) enqueues.  Returns MPI_OK, or the error
    // of a failed capture (the object is then empty; CUDA's sticky-free error
    // state is cleared, so the caller may enqueue the same work directly).
    template <typename F>
    int capture(F &&enqueue)
    {
        if (cudaStreamCreateWithFlags(&cap_, cudaStreamNonBlocking) != cudaSuccess) return fail();
        if (cudaStreamBeginCapture(cap_, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return fail();
        const long long before = counted_launches();
        const int rc = enqueue(cap_);
        uncount_launches(counted_launches() - before);
        const cudaError_t ec = cudaStreamEndCapture(cap_, &graph_);
        if (rc != MPI_OK || ec != cudaSuccess || !graph_) return fail();
        if (cudaGraphGetNodes(graph_, nullptr, &nodes_) != cudaSuccess) return fail();
        if (cudaGraphInstantiate(&exec_, graph_, 0) != cudaSuccess) return fail();
        return MPI_OK;
    }
    int launch(cudaStream_t st);
    bool ready() const { return exec_ != nullptr; }

  private:
    int fail();
    static long long counted_launches();
    static void uncount_launches(long long n);
    cudaStream_t cap_ = nullptr;
    cudaGraph_t graph_ = nullptr;
    cudaGraphExec_t exec_ = nullptr;
    size_t nodes_ = 0;
};

}  // namespace mpi
