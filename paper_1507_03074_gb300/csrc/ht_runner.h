// Runner: the device side of a batch of events, shared by the batch ABI
// (ht_batch.cu) and the server (ht_server.cu).  Internal.
//
// A runner owns an Engine for up to max_events events, fixed staging for
// max_hits hits (x | y | z) and max_events + 1 hit offsets, and the peak
// outputs.  One run: hit copies into the staging, the kernels of steps 1
// and 2 (replayed from a CUDA graph captured per event count and output
// place), then the results: either into device buffers, or written by the
// order kernel straight into mapped pinned host memory (no copy back).
#pragma once

#include <string>
#include <vector>

#include "ht_engine.h"

namespace hte {

struct Runner {
    Engine E;
    uint32_t capacity = 0;           // peaks over one run (compact list)
    float *d_xyz = nullptr;          // staging: x | y | z, max_hits each
    float *h_xyz = nullptr;          // pinned
    uint32_t *d_off = nullptr;       // max_events + 1 hit offsets
    uint32_t *h_off = nullptr;       // pinned
    htk::Peak *d_out = nullptr;      // device outputs
    uint32_t *d_counts = nullptr;
    htk::Peak *h_out = nullptr;      // mapped pinned outputs (written by the order kernel)
    uint32_t *h_counts = nullptr;    // max_events counts + the status word
    htk::Peak *h_out_dev = nullptr;  // their device addresses
    uint32_t *h_counts_dev = nullptr;
    struct Graph {
        uint32_t n_events;
        bool to_host;
        uint32_t fill_flags;         // HT_PEAKS_ONLY, HT_FILL_NAIVE or 0
        cudaGraphExec_t exec;
    };
    std::vector<Graph> graphs;
    bool graphs_ok = true;           // capture works here
};

ht_status runner_create(Runner &R, const ht_binning *b, const ht_ranges *r, uint32_t threshold, uint32_t max_events,
                        uint32_t max_hits, uint32_t capacity, std::string *why);
void runner_destroy(Runner &R);
void runner_drop_graphs(Runner &R);

// Enqueue one run of n_events events on st.  The hits are in the pinned
// staging (host_in) or in the device staging already; the offsets likewise.
// to_host: peaks and counts into the mapped pinned outputs, plus the status
// word into h_counts[max_events]; else into d_out / d_counts.  fill_flags:
// HT_PEAKS_ONLY (the fill keeps its tiles in shared memory, M_H is not
// written; the edge rows must have been allocated, engine_ensure_edges),
// HT_FILL_NAIVE (the paper's fill: clear, one global atomic per vote) or 0.
cudaError_t runner_enqueue(Runner &R, uint32_t n_events, uint32_t n_hits, bool host_in, bool to_host,
                           cudaStream_t st, uint32_t fill_flags = 0);

// After a failed status word: zero the counters (stream-ordered) and map the
// status bits to an ABI code and message.
ht_status runner_status(Runner &R, uint32_t status, cudaStream_t st, std::string *why);

} // namespace hte
