// Filter applications as CUDA graphs: the launch sequence of one call (its
// n_p step kernels per block, the weights, the prepared values, the moment
// finalisation) captured once into a graph and replayed for every later
// call with the same arguments, instead of being launched kernel by kernel.
#include <cstring>
#include <mutex>
#include <vector>

#include "filter.cuh"

namespace cfd {

namespace {

constexpr int kMaxGraphs = 16;        // cached executables (oldest evicted)
constexpr int kMaxDevices = 64;

struct Entry {
    int dev;
    std::vector<char> key;
    cudaGraphExec_t exec;
    long long kernels;                 // kernel launches the graph holds
    unsigned long long last_use;
};

std::mutex g_mu;
std::vector<Entry> g_cache;
unsigned long long g_tick = 0;
cudaStream_t g_capture[kMaxDevices] = {nullptr};

}  // namespace

cfd_status run_as_graph(const void *key, size_t key_bytes, cudaStream_t stream,
                        const std::function<cfd_status(cudaStream_t)> &body) {
    int dev = 0;
    CFD_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return fail(CFD_ERR_ARG, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_mu);
    for (auto &e : g_cache) {
        if (e.dev == dev && e.key.size() == key_bytes && std::memcmp(e.key.data(), key, key_bytes) == 0) {
            e.last_use = ++g_tick;
            CFD_CUDA(cudaGraphLaunch(e.exec, stream));
            count_launches(e.kernels);
            return CFD_OK;
        }
    }
    // capture on the library's own stream of this device (never used
    // otherwise, so it holds no work of its own); relaxed mode: the
    // launchers' occupancy and attribute queries are not stream work
    if (!g_capture[dev]) CFD_CUDA(cudaStreamCreateWithFlags(&g_capture[dev], cudaStreamNonBlocking));
    cudaStream_t cs = g_capture[dev];
    const unsigned long long n0 = launch_count();
    CFD_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed));
    const cfd_status st = body(cs);
    cudaGraph_t graph = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(cs, &graph);
    const long long kernels = (long long)(launch_count() - n0);
    count_launches(-kernels);          // captured, not run yet
    if (st != CFD_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    if (ce != cudaSuccess || !graph)
        return fail(CFD_ERR_CUDA, "stream capture of the filter failed: %s", cudaGetErrorString(ce));
    cudaGraphExec_t exec = nullptr;
    const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) return fail(CFD_ERR_CUDA, "graph instantiation failed: %s", cudaGetErrorString(ie));
    if ((int)g_cache.size() >= kMaxGraphs) {
        size_t old = 0;
        for (size_t i = 1; i < g_cache.size(); ++i)
            if (g_cache[i].last_use < g_cache[old].last_use) old = i;
        cudaGraphExecDestroy(g_cache[old].exec);       // freed once any launch of it completes
        g_cache.erase(g_cache.begin() + (long)old);
    }
    Entry e{dev, std::vector<char>(static_cast<const char *>(key), static_cast<const char *>(key) + key_bytes), exec,
            kernels, ++g_tick};
    g_cache.push_back(std::move(e));
    CFD_CUDA(cudaGraphLaunch(exec, stream));
    count_launches(kernels);
    return CFD_OK;
}

}  // namespace cfd
