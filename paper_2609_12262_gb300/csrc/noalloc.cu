// noalloc.cu -- qec_decode_batch_static: the batched decoder with its scratch
// memory in a fixed file-scope device array instead of a workspace obtained
// from cudaMalloc.
//
// Some callers cannot allocate device memory once they are running: a
// real-time decoding loop in a quantum-control stack must not stall on the
// driver's allocator (cudaMalloc / cudaFree can synchronise the device and take
// milliseconds) or fail half-way for lack of memory, and an application that
// reserves all device memory up front at start-up has nothing left to give
// later.  For them this entry point uses only what the library already holds:
// one static device array of QEC_STATIC_SCRATCH_BYTES (80 MiB) that every GPU
// loading the library keeps until the process exits.  The caller still passes
// the inputs and the outputs.
//
// The array holds, in order: the work counters (zeroed by every call), the
// overflow list of the main pass, and QEC_STATIC_WARPS per-warp slabs sized
// for at most QEC_STATIC_MAX_EVENTS detection events per shot.  Every call
// shares it, so calls whose work overlaps on the GPU (for example on two
// streams of one device) corrupt each other's scratch; the caller must order
// them.  Shots with more detection events than the slab
// holds end with status QEC_SHOT_CAPACITY (there is no second, larger pass).

#include <cstring>
#include <mutex>
#include <string>

#include "qec_internal.h"

namespace {

constexpr long long kScratchBytes = QEC_STATIC_SCRATCH_BYTES;
constexpr int kWarps = QEC_STATIC_WARPS;
constexpr int kKcap = QEC_STATIC_MAX_EVENTS;
constexpr long long kQueueBytes = 256;
constexpr long long kOverflowBytes = (long long)QEC_STATIC_MAX_SHOTS * 4;

static __device__ __align__(256) char g_static_scratch[QEC_STATIC_SCRATCH_BYTES];

struct DevState {
    bool ready = false;
    char *base = nullptr;   // device address of g_static_scratch on this device
};

DevState g_state[64];
std::mutex g_mu;

int err(int code, const std::string &m) { return qec::set_last_error(code, m.c_str()); }

}  // namespace

extern "C" {

int qec_decode_batch_static(const qec_graph *const *graphs, int32_t num_graphs, const int32_t *graph_of_shot,
                            const int64_t *syn_offset_words, const uint32_t *syndromes, int64_t num_shots,
                            uint64_t *obs_out, int64_t *weight_out, int32_t *status_out,
                            qec_cuda_stream stream) {
    if (num_shots < 0) return err(QEC_EINVAL, "num_shots < 0");
    if (num_shots > QEC_STATIC_MAX_SHOTS)
        return err(QEC_ERANGE, "num_shots exceeds QEC_STATIC_MAX_SHOTS (1048576) for the static-scratch decoder");
    if (num_shots == 0) return QEC_OK;
    if (!graphs || num_graphs < 1 || num_graphs > QEC_MAX_GRAPHS_PER_BATCH)
        return err(QEC_EINVAL, "num_graphs out of range");
    if (!syndromes || !obs_out || !weight_out || !status_out) return err(QEC_EINVAL, "NULL buffer");
    int dev = 0;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce != cudaSuccess) return err(QEC_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(ce));
    if (dev < 0 || dev >= 64) return err(QEC_EINVAL, "device index");
    qec::BatchArgs a;
    std::memset(&a, 0, sizeof(a));
    for (int i = 0; i < num_graphs; i++) {
        if (!graphs[i]) return err(QEC_EINVAL, "NULL graph");
        int gdev = -1;
        if (qec::graph_device_view(graphs[i], &a.g[i], &gdev) != QEC_OK || gdev != dev)
            return err(QEC_EINVAL, "graph lives on another device");
    }
    const qec::SlabCaps caps = qec::caps_for_kcap(kKcap);
    const long long slab = qec::slab_bytes_for(caps);
    if (kQueueBytes + kOverflowBytes + slab * kWarps > kScratchBytes)
        return err(QEC_ERANGE, "static scratch too small for its slabs");
    const cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    char *base = nullptr;
    {
        // set-up, once per device, with that device current: look up the
        // array's device address, then fill the slabs with all-ones (empty
        // table entries, which the kernel expects and leaves behind).  The
        // device counts as set up only once that fill is enqueued, so a failed
        // first call is repeated in full by the next one.
        std::lock_guard<std::mutex> lk(g_mu);
        DevState &s = g_state[dev];
        if (!s.ready) {
            cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
            ce = cudaStreamIsCapturing(st, &cs);
            if (ce != cudaSuccess)
                return err(QEC_ECUDA, std::string("cudaStreamIsCapturing: ") + cudaGetErrorString(ce));
            if (cs != cudaStreamCaptureStatusNone)
                return err(QEC_EINVAL, "the first qec_decode_batch_static call on a device must not be captured");
            void *p = nullptr;
            ce = cudaGetSymbolAddress(&p, g_static_scratch);
            if (ce != cudaSuccess || !p)
                return err(QEC_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(ce));
            ce = cudaMemsetAsync(static_cast<char *>(p) + kQueueBytes + kOverflowBytes, 0xff,
                                 (size_t)(slab * kWarps), st);
            if (ce != cudaSuccess) return err(QEC_ECUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(ce));
            s.base = static_cast<char *>(p);
            s.ready = true;
        }
        base = s.base;
    }
    auto *queue = reinterpret_cast<unsigned long long *>(base);
    ce = cudaMemsetAsync(queue, 0, 4 * sizeof(unsigned long long), st);   // counters start at zero
    if (ce != cudaSuccess) return err(QEC_ECUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(ce));
    const qec_tuning tune = qec::current_tuning();
    a.num_graphs = num_graphs;
    a.band_factor = tune.band_factor > 0 ? tune.band_factor : 1;
    a.num_shots = num_shots;
    a.max_events = tune.max_events > 0 ? tune.max_events : 4000000;
    a.graph_of_shot = graph_of_shot;
    a.syn_off = reinterpret_cast<const long long *>(syn_offset_words);
    a.syn = syndromes;
    a.obs_out = reinterpret_cast<unsigned long long *>(obs_out);
    a.w_out = reinterpret_cast<long long *>(weight_out);
    a.st_out = status_out;
    a.queue = queue;
    a.overflow = reinterpret_cast<int *>(base + kQueueBytes);
    a.slabs = base + kQueueBytes + kOverflowBytes;
    a.slab_bytes = slab;
    a.caps = caps;
    a.pass = 0;
    a.single_shot = -1;
    a.watchdog_ns = 60LL * 1000 * 1000 * 1000;
    // one warp per block, so that the persistent warps spread over every SM
    ce = qec::launch_batch(a, kWarps, 32, st);
    if (ce != cudaSuccess) return err(QEC_ECUDA, std::string("kernel launch: ") + cudaGetErrorString(ce));
    return QEC_OK;
}

}  // extern "C"
