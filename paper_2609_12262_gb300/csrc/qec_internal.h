// Internal declarations shared by the host library (capi.cpp) and the CUDA
// kernels (decoder.cu).  Not part of the public ABI.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/qec.h"

namespace qec {

// One CSR slot of a detector, 8 bytes (one vector load): `code` is the
// neighbour detector, or -1 - (merged edge id) for the edge to a boundary
// vertex; `w` is the internal weight (2w).  Merged ids of detector-detector
// slots live in DGraph::seid (read only to trace internal observables).
struct __align__(8) Slot {
    int code;
    int w;
};

// Device view of one graph, passed to kernels by value.
struct DGraph {
    int n;             // detectors
    int words;         // padded uint32 words per syndrome row
    int wmax;          // largest internal weight
    int d1, b1;        // Algorithm 3 level-1 diameter / buffer (internal units)
    int internal_obs;  // some detector-detector edge carries an observable
    int hop2;          // 3 x smallest internal weight > b1: a path of length <= b1 has at most two edges
    int wmin;          // smallest internal weight
    const int *row;                   // [n + 1]
    const Slot *slot;                 // [row[n]]
    const unsigned long long *eobs;   // [merged edges]
    const int2 *eend;                 // [merged edges]: (lower detector endpoint, internal weight)
    const int *seid;                  // [row[n]]: merged edge id of every slot
    const unsigned *commit;           // [words]: detectors of the commit region (sliding windows), or NULL
};

// Capacities of one warp's slab (per-shot working set).
struct SlabCaps {
    int kc;    // detection events
    int hc;    // explored-entry hash slots (power of two)
    int ec;    // explored-entry list
    int wc;    // relaxation work list
    int phc;   // pair hash slots (power of two)
    int nc;    // matcher nodes
    int cc;    // blossom cycle pool
    int wcap;  // syndrome words per row
};

struct BatchArgs {
    DGraph g[QEC_MAX_GRAPHS_PER_BATCH];
    int num_graphs;
    int band_factor;
    long long num_shots;
    long long max_events;
    const int *graph_of_shot;
    const long long *syn_off;
    const unsigned *syn;
    unsigned long long *obs_out;
    long long *w_out;
    int *st_out;
    char *slabs;
    long long slab_bytes;
    SlabCaps caps;
    unsigned long long *queue;   // [0] next work item, [1] overflow count
    int *overflow;               // shot ids that overflowed the main pass
    int pass;                    // 0: all shots, 1: shots listed in overflow
    long long single_shot;       // >= 0: decode only this shot (plain path)
    const int *order;            // pass 0 work order (shot indices), or NULL for 0, 1, 2, ...
    long long watchdog_ns;       // > 0: shots still running this long after the launch stop (budget status)
    int mode;                    // QEC_MODE_HIERARCHICAL or QEC_MODE_GLOBAL
    int *diag_out;               // [num_shots][QEC_DIAG_FIELDS] per-shot counters, or NULL
    // sliding-window mode (carry != NULL): the committed observable is XORed
    // into cobs[shot], the detectors flipped for the next window go to the
    // shot's carry row (same layout as its syndrome row), statuses only ever
    // change to a failure, and obs_out / w_out are not written
    unsigned long long *cobs;
    unsigned *carry;
    // multi-warp teams: a shot with fewer detection events than this is
    // decoded by the team's first warp alone (0: always by the whole team)
    int team_split;
    // serving: per-shot completion flags in host memory mapped into the
    // device (obs_out / w_out / st_out then point there too); set to 1, after
    // a system-wide fence, once a shot's final results are written, or NULL
    int *done;
};

long long slab_bytes_for(const SlabCaps &c);
// Slab capacities for `kcap` detection events; hash tables and entry lists get
// table_factor times the default room per event.
SlabCaps caps_for_kcap(int kcap, int table_factor = 1);
// Team sizes compiled besides one warp per shot: a whole block of TEAM_MID or
// TEAM_BIG warps decodes one shot (large windows, single-window latency).
constexpr int TEAM_MID = 4;
constexpr int TEAM_BIG = 16;
// Launch the batch kernel: team 1 = one warp per shot (grid x block threads),
// TEAM_MID / TEAM_BIG = one block of that many warps per shot (grid blocks);
// sliding-window batches (a.carry set) take team 1 or TEAM_BIG.
cudaError_t launch_batch(const BatchArgs &a, int grid, int block, cudaStream_t s, int team = 1);
// Resident blocks per SM of the multi-warp batch kernel of team size `team`.
int team_occupancy_blocks(int team);
cudaError_t launch_reset_queue(unsigned long long *queue, cudaStream_t s);
// Window syndromes from stream syndromes: bit i of window row r is bit
// (bit_begin + i) of stream row r for i < nbits, XOR bit (carry_begin + i) of
// carry row r for i < carry_bits (carry may be NULL); rows are padded with zeros.
cudaError_t launch_window_assemble(const unsigned *src, long long src_words, long long bit_begin, int nbits,
                                   const unsigned *carry, long long carry_words, long long carry_begin,
                                   int carry_bits, unsigned *dst, long long dst_words, long long num_rows,
                                   cudaStream_t s);
// Order the shots of a mixed batch by graph (graphs in the order given by
// gorder[0 .. ng)), so that concurrently running warps share one graph; gcnt
// holds 64 ints of scratch.
cudaError_t launch_graph_sort(const int *graph_of_shot, long long n, int ng, const int *gorder, int *gcnt,
                              int *order, cudaStream_t s);
// Resident blocks per SM of the batch kernel at this block size.
int occupancy_blocks(int block_threads);
// Largest block the batch kernel accepts.
int max_block_threads();
// Device view and device id of a created graph (QEC_EINVAL for NULL).
int graph_device_view(const qec_graph *g, DGraph *out, int *device);
// The tuning knobs currently set by qec_set_tuning (band width and event
// budget apply to every batched entry point).
qec_tuning current_tuning();
// Record the calling thread's error text for qec_last_error; returns code.
int set_last_error(int code, const char *msg);

}  // namespace qec
