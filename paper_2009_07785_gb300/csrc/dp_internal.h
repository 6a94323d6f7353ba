// Internal types shared by the library's host and device sources.
//
// Device layout of a loaded matrix ("sliced ELL over row chunks"):
//   Every row is cut into chunks of at most `chunk` nonzeros (a row that
//   fits is one chunk).  Chunks of rows that had to be split ("split rows")
//   come first, sorted by length; the remaining single-chunk rows follow,
//   sorted by length, longest first.  32 consecutive chunks form a slice,
//   which one warp processes with one chunk per lane.  A slice stores its
//   nonzeros slot-major: element (slot k, lane t) of slice s sits at
//   slice_off[s] + 32*k + t, so the 32 lanes read 32 consecutive values and
//   32 consecutive column indices per slot.  Within a chunk the slots keep
//   the row's CSR order.
//
// Merge-path layout (an alternative to the above; the paper's Conclusions
// and Outlook name newer SpMV algorithms than CSR-adaptive as a direction
// for computing activities): rows, grouped by side class, in
// plain CSR; the sequence of m row ends and nnz nonzeros (merged in CSR
// order) is cut into segments of `mp_ipt` items, one per thread, so every
// thread does equal work whatever the row lengths.  A thread sums the
// nonzeros of its segment sequentially row by row; a row that lies inside
// one segment is summed exactly as the CSR order sums it, a row that
// crosses segment boundaries ("split row") is summed in pieces that a
// second pass combines in segment order.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace dp {

// Every device allocation of the library goes through these two (dp_capi.cu):
// they keep a process-wide count of live allocations and can be told to
// fail, for the allocation-failure test hook dp_debug_fail_alloc.
cudaError_t dev_malloc(void **p, size_t bytes);
void dev_free(void *p);
void arm_alloc_failure(int32_t k);  // the k-th allocation from now fails; 0 disarms
int64_t live_allocs();

constexpr int kSliceW = 32;                 // chunks per slice (= warp width)
constexpr int32_t kLenMask = 0x3FFFFFFF;    // chunk length bits
constexpr int32_t kExactFlag = 1 << 30;     // row must skip the FP32 screen
constexpr int32_t kLayoutEll = 0;           // sliced ELL over row chunks
constexpr int32_t kLayoutMerge = 1;         // merge-path segments over CSR
// A block of the persistent loop waits at a grid barrier for at most this
// many 64 ns sleeps (about 2 s) before it records DP_ERR_TIMEOUT and leaves.
constexpr long long kDefaultWaitLimit = 1ll << 25;

// Current bounds of one variable, as gathered by the round kernels: one
// 32-byte record, fetched with a single 256-bit load per nonzero.
struct alignas(32) VarRec {
  double L, U;     // bounds at the start of the round
  float WU, WL;    // screen widths for upper / lower candidates (see kernels)
  uint32_t flags;  // bit 0: integer variable
  uint32_t pad;
};
static_assert(sizeof(VarRec) == 32, "VarRec must be one 32-byte sector");

// Partial activity of one chunk of a split row.
// Screen values of a chunk, per side: the largest (T1) and second largest
// (T2) upper bounds on |a| W over the chunk, and the slot of the largest.
// Also the slot of an infinite contribution to each activity (the one that
// gets a finite residual when the row has exactly one, Sec. 3.4).
struct Top2 {
  float r1, r2, l1, l2;
  int32_t kr, kl;
  int32_t kinf_min, kinf_max;
};

struct alignas(16) Partial {
  double minfin, maxfin;
  int32_t mininf, maxinf;
  Top2 t;
  int32_t exact;    // the chunk's row must skip the FP32 screen
  int32_t pad;
};

// Combined activity of one split row, plus the screen thresholds.
struct alignas(16) RowTot {
  double minfin, maxfin;
  int32_t mininf, maxinf;
  float thr_r, thr_l;  // a nonzero with |a| W <= thr cannot tighten from that side
  int32_t active;      // some nonzero of the row may yield an accepted candidate
  int32_t row;
};

// One nonzero whose candidates survived the screen, queued for the
// lane-dense candidate kernel: its element offset in val/col, and
// (chunk slot << 2 | sides), sides bit 0 = right-hand side, bit 1 = left.
// The queue holds one entry per slot at most, so it cannot overflow.
struct alignas(8) CandEntry {
  uint32_t off;
  uint32_t cs;
};

// Activity sums of the row a queued chunk belongs to (written by the lane
// that queues the chunk's first survivor; indexed by chunk slot).
struct alignas(8) RowSum {
  double minfin, maxfin;
  int32_t mininf, maxinf;
};

// Device control block of one propagation run.
struct Ctrl {
  int32_t round;        // executed rounds
  int32_t max_rounds;
  int32_t changed;      // a candidate was accepted in the current round
  int32_t last_changed; // value of `changed` at the end of the last round
  int32_t infeasible;
  int32_t err;          // 0, or a DP_ERR_* code found by the prologue
  uint32_t blocks_done; // arrival counter of the last kernel of a round
  int32_t qcount;       // entries appended to the candidate queue this round
  int32_t cont;         // the last round asked for another one
  int32_t pad;
  double eps_int, tau_rel, eps_feas, inf_thr;
  long long wait_limit;  // persistent loop: sleeps a block waits at a grid barrier
};

struct DevMatrix {
  int32_t m, n;
  int64_t nnz;
  int32_t nslices;        // all slices
  int32_t nslices_split;  // slices [0, nslices_split) hold split-row chunks
  int32_t nsplit_rows;
  int32_t round_warps;      // warps per block of the round kernel (4 or 8)
  const double *val;        // padded slot-major values
  const int8_t *val8;       // the same values as int8 when all are small
                            // integers and compression is on, else null
  const int32_t *col;       // padded slot-major column indices
  const int64_t *slice_off; // [nslices] element offset of each slice
  const int32_t *slice_len; // [nslices] slots in each slice
  const int32_t *chunk_row; // [nslices*32] row of each chunk, -1 = padding
  const int32_t *chunk_len; // [nslices*32] length | kExactFlag
  const int32_t *chunk_sidx;// [nslices_split*32] split-row index, -1 = none
  const int32_t *split_row; // [nsplit_rows] row id of each split row
  const int32_t *split_cbeg;// [nsplit_rows+1] range of each split row in split_cidx
  const int32_t *split_cidx;// chunk slots of the split rows' pieces, row by row
                            // (merge path: piece indices, 2t = head of
                            // segment t, 2t+1 = its carry)
  // merge-path layout only (layout == kLayoutMerge; val/col then hold the
  // rows' CSR in side-class order, chunk_row maps that order to the
  // caller's rows and chunk_len holds row length | kExactFlag)
  int32_t layout;           // kLayoutEll or kLayoutMerge
  int32_t mp_ipt;           // items (row ends + nonzeros) per segment
  int32_t mp_nseg;          // segments (threads)
  int32_t mp_pad;
  const int32_t *mp_ptr;    // [m+1] CSR row offsets in side-class order
  const int32_t *mp_srow;   // [mp_nseg+1] rows whose end precedes each segment
  // rows longer than kMpLaneRow ("long rows"; chunk_sidx[p] = their index)
  // are re-read for the screen by one warp per piece of <= kMpPiece nonzeros
  int32_t mp_nlong, mp_npiece;
  const int4 *mp_piece;     // [mp_npiece] {row, long index, CSR offset, length}
};
constexpr int32_t kMpLaneRow = 64;  // longest row whose screen one lane re-reads
constexpr int32_t kMpPiece = 256;   // nonzeros per warp in the long-row re-read

// Several independent problems in one matrix (their block-diagonal union:
// each problem owns its rows and variables) with per-problem termination.
// All pointers are null for a single problem.
struct InstState {
  const int32_t *slot_inst;  // [chunk slots] problem of each chunk's row
  const int32_t *var_inst;   // [n] problem of each variable
  int32_t *changed;          // [ninst] a candidate was accepted this round
  int32_t *infeasible;       // [ninst]
  int32_t *done;             // [ninst] stopped: no change, infeasible or the cap
  int32_t *rounds;           // [ninst] executed rounds
  int32_t *status;           // [ninst] 1 = stopped by the cap
  int32_t ninst;
  int32_t pad;
};

struct DevState {
  CandEntry *queue;     // [padded slots] candidate queue
  RowSum *rowsum;       // [chunk slots] sums of rows with queued nonzeros
  VarRec *rec;          // [n] state at the start of the round
  long long *keys;      // [2n] next state as order-preserving int64 keys
  double *lhs, *rhs;    // [m] normalised sides
  double2 *side;        // [chunk slots] {lhs, rhs} of each chunk's row, in slot order
  Partial *part;        // [nslices_split*32]
  RowTot *rowtot;       // [nsplit_rows] (merge path: [mp_nlong], long rows)
  Partial *rowact;      // merge path: [m] activities of each row (side-class order)
  uint32_t *mp_need;    // merge path: [ceil(mp_nseg/32)] activities a warp's rows need
  Ctrl *ctrl;
  uint32_t *dirty;      // [ceil(n/32)] bit j: x_j's next state changed this round
  unsigned *bar;        // [2] grid barrier of the persistent loop: arrivals, generation
  InstState I;          // problem sets only
};

// ------------------------------------------------------ batched B&B nodes --
//
// One batched call propagates Bp = 32*G bound vectors ("nodes") over one
// matrix.  Bounds are stored node-minor, entry e = j*Bp + node, so that the
// 32 lanes of a warp (32 nodes of one node group g) read the bounds of one
// variable with one 512-byte coalesced load, while the matrix row is read
// once per warp with warp-uniform loads.
constexpr int kMaxGroups = 32;              // at most 1024 nodes per launch

// Partial activity of one chunk of a split row for one node.
struct alignas(16) BPartial {
  double minfin, maxfin;
  int32_t mininf, maxinf;
  float tr, tl;   // largest screen values of the chunk (right / left side)
};

// Combined activity of one split row for one node, with its screen
// thresholds (a nonzero with |a| W <= thr cannot tighten from that side).
struct alignas(16) BRowTot {
  double minfin, maxfin;
  int32_t mininf, maxinf;
  float thr_r, thr_l;
};

struct BCtrl {
  int32_t round;      // executed rounds
  int32_t max_rounds;
  int32_t B;          // real nodes
  int32_t Bp;         // padded nodes (32*G)
  int32_t G;          // node groups
  int32_t err;        // 0, or a DP_ERR_* code found by the prologue
  int32_t any_alive;  // some node is still propagating
  uint32_t blocks_done;
  uint32_t bar_count;    // persistent loop: grid-barrier arrivals
  uint32_t bar_gen;      //   and its generation
  long long wait_limit;  // persistent loop: sleeps a block waits at a grid barrier
  int32_t icount[kMaxGroups];  // work items of each node group this round
  double eps_int, tau_rel, eps_feas, inf_thr;
};

struct BatchState {
  double2 *cur;         // [n*Bp] {L, U} at the start of the round
  float2 *wid;          // [n*Bp] screen widths {W_U, W_L} of those bounds
  long long *nkey;      // [2*n*Bp] next state as order-preserving keys
  uint32_t *chg[2];     // [n*Gs] nodes of each group whose bounds of var j changed
                        // (set while a round runs, committed and cleared after)
  uint32_t *cmask;      // [nslots*G] nodes of each group that process a chunk
  int32_t *items;       // [G*nslots] chunk slots to process, one region per group
  BPartial *part;       // [nsplit_slots*Bp]
  BRowTot *rowtot;      // [nsplit_rows*Bp]
  uint32_t *srow_act;   // [nsplit_rows*G] nodes whose split row yields candidates
  uint32_t *inf_bits;   // [kMaxGroups] nodes whose infeasibility was detected
  uint32_t *chg_bits;   // [kMaxGroups] nodes with a changed bound this round
  int32_t *node_rounds; // [Bp] rounds executed for the node
  int32_t *node_status; // [Bp] 1 = stopped by the round cap
  int32_t *node_done;   // [Bp]
  uint32_t *alive;      // [G] nodes still propagating
  uint32_t *fresh;      // [kMaxGroups] nodes in their first round (every row active)
  double *lhs, *rhs;    // [m] normalised sides
  uint8_t *vt;          // [n] 0/1 variable types
  BCtrl *ctrl;
  int64_t nslots;       // chunk slots (the capacity of one item region)
};

}  // namespace dp
