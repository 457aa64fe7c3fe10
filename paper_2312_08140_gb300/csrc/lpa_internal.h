// lpa_internal.h -- layout of the device-resident state of one label
// propagation engine and the launchers the host code calls.  Shared by the
// kernel translation units and the C-ABI implementation; not installed.
//
// One engine runs G >= 1 independent graphs packed into one CSR with global
// vertex ids (a single graph is G = 1).  Per sweep t (lpaMove of Algorithm 1):
//   sweep kernels  (one per degree bin) read the frontier lists L_t, pick the
//                  most weighted label per vertex (Eq. 2, smallest-id ties),
//                  write changes and re-flag neighbours (vertex pruning);
//   finish kernel  applies the sync-mode changes, compacts flags into L_{t+1}
//                  and, in its last block, runs the per-graph tolerance test
//                  of Algorithm 1 and sets the device-side loop condition.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

namespace lpa {

constexpr int kMaxHist = 64;            // per-sweep history depth (LPA_MAX_RECORDED_ITERS)
constexpr int kBins = 5;                // thread / warp / 128-, 256-, 512-thread block per vertex
constexpr int kBlockBins = 3;           // bins 2..4 use the block kernel
constexpr int kBlockThreads[kBlockBins] = {128, 256, 512};
constexpr int kHighPermille = 900;      // "almost every vertex changed" (see skip_marks)
constexpr int kSliceLen = 4096;         // entries per slice of an overflowing row
constexpr int kMaxParts = 4096;         // partitions a row may use on the sliced path
constexpr int kMaxSlices = 4096;        // slices a row may use on the sliced path (with the above: d <= 2^24)
constexpr int kSliceMinParts = 2;       // every overflowing row (>= 2 partitions) takes the sliced path
                                        // within its limits; the rescan path takes the rest
constexpr int kLargeSlots = 8192;       // shared table of the last bin (overflowing rows are
                                        // rescanned split over label partitions)
constexpr int32_t kEmptyKey = -1;       // free slot in label tables; labels are >= 0

// Tolerance test of Algorithm 1 (Section 4.1.3), dN / N <= tau, as one
// integer threshold per graph: a sweep with dN <= floor(tau * N) meets it,
// the product rounded once to fp64.  IEEE round-to-nearest multiplication
// gives the same threshold on the host and on the device.
__host__ __device__ inline long long dn_threshold(double tau, long long n) {
    return (long long)floor(tau * (double)n);
}

// Weight storage: none (unit weights), integer weights as uint32 or, when all
// are at most 255, as uint8 (sums are uint32 in both), or float.
enum WeightKind : int { W_UNIT = 0, W_U32 = 1, W_F32 = 2, W_U8 = 3 };
enum Mode : int { MODE_SYNC = 0, MODE_ASYNC = 1, MODE_SYNC_FULL = 2 };
// OR'd into the mode passed to the sweep launchers: instantiate the
// non-strict tie-break (compile-time, so the strict kernels are unchanged).
constexpr int kModeNonstrict = 8;

// Control block, one per engine, in device memory.
struct Ctrl {
    int32_t iter;                        // sweeps completed so far (t)
    int32_t max_iters;
    double tau;
    int32_t mode;
    int32_t any_active;                  // loop condition mirror (read by the profiled path)
    int32_t* labels_out;                 // destination of the finalize kernel
    int32_t local_ids;                   // finalize writes label - first vertex of its graph
    int32_t error;                       // non-zero: a device-side check failed
    unsigned int ticket;                 // last-block election in the finish kernel
    int32_t rd;                          // frontier buffer the sweep kernels read (flipped by
                                         // every compaction, which writes buffer rd ^ 1)
    int32_t dense[2];                    // buffer holds the static bin lists (every vertex)
    int32_t cbuf;                        // labels of the current sweep are lab[cbuf]
    int32_t allow_dense;                 // 0: every pass compacts the marks (serving arena)
    int32_t skip_marks;                  // current pass writes no neighbour marks; the next
                                         // pass is dense (scans every vertex) instead
    int32_t last_pass_high;              // previous pass changed >= kHighPermille of entries
    unsigned int bin_cnt[2][kBins];      // frontier list lengths per buffer
    unsigned long long bin_entries[2][kBins];   // CSR entries of those vertices
    unsigned long long bin_changed[kBins];      // vertices changed in the current sweep, per bin
    unsigned long long bin_changed_entries[kBins];
    unsigned long long pass_changed_entries;    // entries of vertices changed since the last compaction
    long long sweep_bin_vertices[kBins];        // scanned in the current sweep (all passes)
    long long sweep_bin_entries[kBins];
    long long hist_active[kMaxHist];
    long long hist_scanned[kMaxHist];
    long long hist_bin_vertices[kMaxHist][kBins];
    long long hist_bin_entries[kMaxHist][kBins];
    long long hist_bin_changed[kMaxHist][kBins];
    long long hist_changed_entries[kMaxHist];
    long long hist_bin_changed_entries[kMaxHist][kBins];
    long long total_sweeps;              // cumulative over all runs (never reset)
    long long total_scanned;
    long long total_sweep_launches;      // kernel launches of those sweeps
    int32_t nonstrict;                   // non-strict tie-break for this run (Section 4.1.5)
    int32_t prune_other;                 // async: a changed vertex marks only neighbours not in its new label
    unsigned long long ovf_count;        // overflow rows appended in this pass
    unsigned int ovf_slice_items;        // work items of the overflow kernels (set by k_ovf_plan)
    unsigned int ovf_part_items;
    unsigned int ovf_rescan_items;
    int32_t stall_copy;                  // test hook (lpa_graph_debug_stall): the block size of the
                                         // row kernel whose first block to produce a tile leaves that
                                         // tile's index copy unissued, once
    unsigned int row_next[kBins];        // block bins: next list position to take in this pass
    unsigned int row_next_pad[8 - kBins];
};

// A last-bin row whose labels overflowed the shared table in this pass.  Its
// labels are split over `parts` hash partitions; each partition's block folds
// its best (sum, label) into `best` and the block that completes the row
// applies the result.
// Sliced path (kSliceMinParts <= parts <= kMaxParts, scratch available): blocks over
// kSliceLen-entry slices group the row's labels by hash partition into
// scratch, then a block per partition aggregates its share.  Rescan path
// (otherwise): a block per partition rescans the whole row.
struct Overflow {
    int32_t v;                 // vertex
    uint32_t slot;             // its slot in the bin's frontier list
    int64_t st;                // row start
    int32_t d;                 // row length
    int32_t own;               // label before the sweep
    uint32_t parts;            // P = ceil(2d / kLargeSlots) label partitions
    uint32_t slices;           // Q = ceil(d / kSliceLen) on the sliced path, else 0
    int64_t pair_base;         // sliced: first (label, sum) pair of its scratch (d reserved)
    int64_t cnt_base;          // sliced: first of its Q x P (slice, partition) counts and offsets
    uint32_t slice_base;       // sliced: first slice work item
    uint32_t part_base;        // sliced: first partition work item
    uint32_t rescan_base;      // rescan: first partition work item
    uint32_t rescan_parts;     // rescan: P, else 0
    unsigned long long best;   // max over partitions of (sum key << 32) | (~label)
    unsigned int done;         // partitions completed
    unsigned int pad;
};

// Everything a kernel needs, passed by value.
struct DevState {
    int64_t N;                 // vertices over all graphs
    int64_t E;                 // CSR entries
    int32_t G;                 // graphs
    int32_t weight_kind;       // WeightKind
    int32_t small_iota;        // dense sync passes of bin 0 walk vertex ids 0..N-1 (bin 0 holds >= 3/4 of them)
    int32_t rows_distinct;     // no row repeats a neighbour: the first synchronous sweep is a max-weight reduction
    const int64_t* off;        // [N] row begins (positions in idx)
    const int64_t* off_end;    // [N] row ends (off + 1 for an ordinary CSR)
    const int32_t* idx;        // [E] global vertex ids
    const void* w;             // [E] uint8 (W_U8), uint32 (W_U32), float (W_F32) or null (W_UNIT)
    const int32_t* gid;        // [N] graph of each vertex, null when G == 1
    const int32_t* orig;       // [N] original (global) id of each stored vertex, null when the vertices
                               // are stored in the caller's order.  Labels are always original ids.
    const int64_t* vtx_off;    // [G+1] (batches)
    const int64_t* g_begin;    // [G] first vertex of graph g (vtx_off for batches)
    const int64_t* g_end;      // [G] one past its last vertex (vtx_off + 1 for batches)
    int32_t* lab[2];           // [N] label buffers (global ids): current lab[cbuf]; sync sweeps write
                               // the other one (every scanned vertex in dense sweeps, then the
                               // buffers flip; only changed vertices in sparse sweeps, then applied)
    uint8_t* flags;            // [N] 1 = unprocessed (Algorithm 1)
    uint16_t* fr_bits;         // [N/16 + 1] async: bit q of word c = vertex 16c + q is in this sweep's
                               // main frontier (written by the sparse compaction that starts a sweep)
    int32_t* slist;            // [N] static lists: vertices with an entry, by bin, ascending
    int32_t* flist;            // [N] frontier lists of the sparse sweeps, same bin regions
    int32_t* chg;              // [N] sync mode, aligned with list slots: vertex if changed, else -1
    int64_t bin_base[kBins];   // first slot of each bin's region in slist / flist / chg
    unsigned int bin_static[kBins];            // vertices of each bin (static list lengths)
    unsigned long long bin_static_entries[kBins];
    int64_t active_entries;    // entries of all vertices with an entry (= E)
    Ctrl* ctrl;
    unsigned long long* dN;    // [G] changed vertices of the current sweep
    int32_t* done;             // [G]
    int32_t* iters;            // [G]
    int32_t* exit_reason;      // [G]
    long long* hist_changed;   // [G * kMaxHist]
    struct Overflow* ovf;      // [bin_static[4]] last-bin rows whose labels overflowed the shared table
    uint2* ovf_pairs;          // sliced path: (label, sum bits) pairs grouped by partition per slice
    uint32_t* ovf_cnt;         // sliced path: pairs per (slice, partition)
    uint32_t* ovf_off;         // sliced path: their offsets within the slice
    int64_t ovf_pairs_cap;     // capacity of ovf_pairs (0: every overflow row takes the rescan path)
    int64_t ovf_cnt_cap;       // capacity of ovf_cnt / ovf_off
    int32_t ovf_possible;      // some last-bin row is longer than kLargeSlots / 2 (else no row overflows)
    int32_t small_max;         // degree bins (see lpa_config)
    int32_t warp_max;
    int32_t mid_max;
    int32_t large_max;
    int32_t warp_slots;        // per-warp table slots = next pow2 >= 2 * warp_max
    int32_t block_slots[kBlockBins];   // per-block shared table slots of bins 2..4
    int32_t dense_permille;    // dense sweep when entries of changed vertices >= this / 1000 of E
};

// ---- launchers (return cudaSuccess or the launch error) ------------------
struct LaunchShape {
    int blocks;
    int threads;
    size_t smem;
};

cudaError_t launch_init(const DevState& s, cudaStream_t st, int sms);
// Static bin lists (slist, bin_base, bin_static*, active_entries) from the
// degrees and the bin limits in s.  Synchronises `st`.
// Static per-bin vertex lists (used by dense sweeps).  counts/ents: device
// scratch of kBins * static_scratch_blocks(N) elements each.
int64_t static_scratch_blocks(int64_t N);
cudaError_t build_static_lists(DevState& s, cudaStream_t st, unsigned* counts, unsigned long long* ents);
// Scratch of the sliced overflow path for the current static lists: pairs and
// (slice, partition) counts it may need, and the number of last-bin rows that
// can overflow at all.  scratch3: device unsigned long long[3].  Synchronises st.
cudaError_t ovf_capacity(const DevState& s, cudaStream_t st, int sms, int64_t* pairs, int64_t* counts,
                         int64_t* rows, unsigned long long* scratch3);
cudaError_t launch_init_cond(const DevState& s, cudaGraphConditionalHandle h, int in_graph, cudaStream_t st);
// Roles of the finish kernel.  A sweep scans each vertex at most once
// (Algorithm 1): the compaction that starts a sweep takes every marked vertex
// and records them in fr_bits; the asynchronous catch-up compaction takes only
// the vertices marked since then that are not in that frontier (the ones the
// serial loop would still reach later in the same sweep); the others keep
// their mark for the next sweep.
enum FinishRole {
    kRoleEndSweep = 0,    // apply, compaction that starts the next sweep, control
    kRoleCatchUp = 1,     // async: compaction of the catch-up set only
    kRoleControl = 2,     // end of a serving cycle: apply, control; marks stay for the next cycle
    kRoleStartSweep = 3,  // start of a serving cycle: compaction (also of newly admitted requests)
};
cudaError_t launch_finish(const DevState& s, int mode, int role, cudaGraphConditionalHandle h, int in_graph,
                          cudaStream_t st, int sms);
cudaError_t launch_finalize(const DevState& s, cudaStream_t st, int sms);
cudaError_t launch_set_params(Ctrl* ctrl, double tau, int max_iters, int mode, int nonstrict, int prune_other,
                              int32_t* labels_out, int local_ids, cudaStream_t st);
cudaError_t launch_sweep_small(const DevState& s, int mode, cudaStream_t st, int sms);
cudaError_t launch_sweep_warp(const DevState& s, int mode, cudaStream_t st, int sms);
// Block-per-vertex sweep of bin 2, 3 or 4 (one resident wave over `sms` SMs).
// For bin 4 this also launches the partitioned rescan of overflowed rows.
cudaError_t launch_sweep_block(const DevState& s, int mode, int bin, int sms, cudaStream_t st);
// The block-per-row kernel of bins 2..4 (lpa_sweep_rows.cu); *blocks receives
// its grid size.
template <bool ASYNC, int WK, bool BATCH, bool NS>
cudaError_t launch_rows(const DevState& s, int bin, int flag, int sms, cudaStream_t st, int* blocks);

// Degree histogram of vertices [0, s.N): kDegBuckets buckets b = ceil(log2 d)
// of vertex counts, then of entry counts (device unsigned long long[2 x
// kDegBuckets], cleared here).
constexpr int kDegBuckets = 40;
cudaError_t launch_degree_hist(const DevState& s, unsigned long long* hist, cudaStream_t st, int sms);

// Storage orders (lpa_reorder.cu): the vertices of a graph may be stored in
// an order of their own while labels stay original ids.
enum StorageOrder : int { kOrderCaller = 0, kOrderDegree = 1, kOrderShuffle = 2 };
// orig[p] (original id of stored vertex p) and inv[v] (stored position of
// original vertex v) for the order; scratch: reorder_scratch_words(N)
// unsigned words.  Synchronises st.
cudaError_t reorder_positions(int kind, const int64_t* off, const int64_t* vtx_off, const int32_t* gid, int32_t G,
                              int64_t N, uint64_t seed, int32_t* orig, int32_t* inv, unsigned* scratch,
                              cudaStream_t st, int sms);
int64_t reorder_scratch_words(int64_t N);
// The CSR in stored order: new_off[N+1], new_idx (neighbours renumbered
// through inv), new_w (wbytes 0, 1 or 4 per entry).  Synchronises st.
cudaError_t reorder_rows(const int32_t* orig, const int32_t* inv, const int64_t* off, const int32_t* idx,
                         const void* w, int wbytes, int64_t N, int64_t* new_off, int32_t* new_idx, void* new_w,
                         unsigned long long* scratch, cudaStream_t st, int sms);

// Graph validation (row-wise).  Results accumulate into *res (device).
struct ValidateResult {
    // c[0] rows with invalid offsets, c[1] indices out of range, c[2] weights
    // negative or not finite, c[3] weights not integer-valued, c[4] rows of
    // weighted degree >= 2^24 (fp32 sums may round), c[5] rows of weighted
    // degree >= 2^31 (32-bit integer sums may overflow)
    unsigned int c[6];
    unsigned long long max_degree;
    unsigned int max_weight_bits;      // bits of the largest valid weight (>= 0, so ordered as unsigned)
    unsigned int pad;
    // single graphs: adjacent entry pairs that do not increase, over all
    // entries and over row starts only; equal <=> every row strictly increases
    unsigned long long desc_all;
    unsigned long long desc_row_starts;
};
// Entry checks of entries [e_begin, e_end) (indices in range, weights finite
// and >= 0, integrality, largest weight, descents; for batches the rewrite of
// local ids to global ones); then, once every entry is in place and checked,
// the row checks (offsets, degrees, exact weighted degrees, descents at row
// starts).  Both accumulate into *res.
cudaError_t launch_validate_entries(const int32_t* idx, const float* w, int64_t N, int64_t E, int64_t e_begin,
                                    int64_t e_end, const int64_t* vtx_off, const int64_t* edge_off, int32_t G,
                                    int rewrite_local_ids, int32_t* idx_rw, ValidateResult* res, cudaStream_t st,
                                    int sms);
cudaError_t launch_validate_rows(const int64_t* off, const int32_t* idx, const float* w, int64_t N, int64_t E,
                                 const int64_t* vtx_off, const int64_t* edge_off, const int32_t* gid, int32_t G,
                                 ValidateResult* res, cudaStream_t st, int sms);
cudaError_t launch_fill_gid(const int64_t* vtx_off, int32_t G, int64_t N, int32_t* gid,
                            cudaStream_t st, int sms);
cudaError_t launch_weights_to_u32(float* w, int64_t E, cudaStream_t st, int sms);
cudaError_t launch_weights_to_u8(const float* w, unsigned char* out, int64_t E, cudaStream_t st, int sms);

// Modularity (Eq. 1), fp64.  Vertex range [v0, v1), labels local to v0.
struct ModAccum {
    double two_m;
    double sigma;
    double null_sum;
    unsigned int bad_label;
    unsigned int pad;
};
cudaError_t launch_modularity(const DevState& s, int64_t v0, int64_t v1, const int32_t* labels,
                              double* Sigma, ModAccum* acc, cudaStream_t st, int sms);

}  // namespace lpa
