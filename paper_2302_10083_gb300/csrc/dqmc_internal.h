// dqmc_internal.h -- host-side plan of the sweep and the launch helpers shared
// by the C ABI (dqmc_api.cu), the sweep kernels (dqmc_sweep.cu) and the
// compaction kernels (dqmc_list.cu).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

namespace dqmc {

// Tile pass kinds.  Every pass works on tiles of 3^K "group" rows x 3^B
// "inner" rows of the padded state (one row = one 32-byte chunk of five
// ternary digits); see dqmc_sweep.cu.
enum PassKind : int {
    kPassFirst = 0,   // read the truth table, Merge chunk digits + group digits
    kPassMerge = 1,   // read rows whose group digits are 0/1, Merge group digits
    kPassReduce = 2,  // read all rows, Reduce group digits
};

struct Pass {
    int kind = kPassFirst;
    int K = 0;              // group digits (high digits a .. a+K-1)
    int B = 0;              // inner digits carried for contiguity (high digits 0 .. B-1)
    int a = 0;              // first group digit (0-based high digit)
    bool top_binary = false;    // digits above the group only take 0/1 (not merged yet)
    bool fuse_reduce = false;   // Merge pass: Reduce the group digits afterwards
    bool chunk_reduce = false;  // Reduce the five chunk digits in this pass
    bool write_out = false;     // write the dense bitmap and the count, not the state
    uint64_t tiles = 0;
    uint64_t n_mid = 1;     // 3^(a-B): assignments of the digits between inner and group
    uint64_t w_g = 1;       // row weight of group digit 0: 3^a
    uint64_t w_top = 1;     // row weight of the first digit above the group: 3^(a+K)
};

// ---------------------------------------------------------------- super-passes
// A super-pass is one persistent kernel launch.  Its rows are split into
// super-blocks (a set of high digits varies inside a block, the others are
// fixed per block); each super-block goes through up to three phases, and each
// phase covers the block with tiles of <= 729 rows (group digits a..a+K-1 and
// inner digits 0..B-1 vary inside a tile).  A tile of phase p > 0 starts only
// after every tile of phase p-1 of its super-block is done, so the block's rows
// stay in L2 between phases.
constexpr int kMaxPhases = 3;
constexpr int kMaxFixed = 24;

enum LoadKind : int { kLoadTT = 0, kLoadSparse = 1, kLoadFull = 2 };

struct FixedDigits {
    int n = 0;
    uint64_t w3[kMaxFixed] = {};    // row weight 3^j of high digit j
    uint64_t w2[kMaxFixed] = {};    // truth-table word weight 2^j (used by kLoadTT)
    uint8_t r[kMaxFixed] = {};      // 2: the digit still takes only 0/1 (not merged yet); 3: any
    uint8_t j[kMaxFixed] = {};      // which high digit (for the plan description)
};

struct PhaseDesc {
    int load = kLoadFull;
    int K = 0, B = 0, a = 0;        // group digits a..a+K-1, inner digits 0..B-1
    int merge = 0;                  // Merge the group digits (kLoadTT: chunk digits first)
    int reduce = 0;                 // Reduce the group digits
    int chunk_mask = 0;             // chunk digits Reduced here (bit i = chunk digit i)
    int out = 0;                    // write the dense bitmap (+ count, + list) instead of rows
    // Neighbour group (out phase only): high digits nbr_a .. nbr_a+nbr_K-1 are
    // also reduced here, each cell against its '*' neighbours in those digits
    // as the previous pass left them in the state (the neighbour tiles are
    // read from device memory; nbr_K = 0: none).
    int nbr_a = 0, nbr_K = 0;
    uint32_t tiles = 1;             // tiles per super-block = product of fix.r
    FixedDigits fix;                // super-block digits fixed per tile
};

struct SuperPassDesc {
    int nph = 1;
    PhaseDesc ph[kMaxPhases];
    uint64_t n_sb = 1;              // super-blocks = product of sb.r
    uint32_t window = 1;            // super-blocks per pipeline step
    FixedDigits sb;                 // digits fixed per super-block
    uint64_t done_off = 0;          // offset (in uint32) of this pass's phase counters
    int slot = 0;                   // ticket counter index
    // Ticket layout: n_steps pipeline steps of step_size tickets; within step
    // k, phase p owns tickets [ph_off[p], ph_off[p] + window * tiles_p) and
    // runs super-block group k - p (tickets of groups outside 0..groups-1, or
    // of super-blocks past n_sb in the last group, are empty).
    uint32_t step_size = 0, n_steps = 0, groups = 0;
    uint32_t ph_off[kMaxPhases] = {};
};

struct Plan {
    int n = 0;
    int C = 0;              // chunk digits: min(n, 5)
    int H = 0;              // high digits: n - C
    uint64_t state_rows = 0;    // rows of the device state (0: the state lives in shared memory)
    std::vector<Pass> passes;           // n <= 12: the one whole-function pass
    std::vector<SuperPassDesc> sps;     // n >= 13: persistent super-passes
    uint64_t n_done = 0;                // phase counters (uint32) over all super-passes
    uint64_t out_tiles = 0;             // tiles of the bitmap phase (look-back slots)
};

constexpr int kMaxSmemGroup = 7;    // 3^7 rows x 32 B = 70 KB of shared memory
constexpr int kMaxStreamGroup = 6;  // digits of a group after the first
constexpr int kTileDigits = 7;      // group + inner digits of a streaming tile
constexpr int kTileRows = 2187;     // 3^7

Plan make_plan(int n);
std::string describe_plan(const Plan &p);
int plan_passes(const Plan &p);     // kernel launches of the sweep

// Workspace layout (offsets in bytes from the workspace base, 256-aligned).
struct Workspace {
    uint64_t state_off = 0, state_bytes = 0;
    uint64_t count_off = 0;             // uint64 scratch counter
    uint64_t ctrl_off = 0, ctrl_bytes = 0;  // error word, tickets, phase counters, look-back slots
    uint64_t blk_counts_off = 0;        // uint32 per compaction block
    uint64_t blk_offs_off = 0;          // uint64 per compaction block
    uint64_t n_blocks = 0;
    uint64_t total = 0;
};
Workspace workspace_layout(int n);

uint64_t bitmap_words(int n);        // ceil(3^n / 32)
uint64_t bitmap_alloc_bytes(int n);  // ceil(3^n / 8) rounded up to 16

// A batch of functions with the same n (device tables, indexed by function
// id): the pass kernels and the one-tile kernel run every function of the
// batch in one launch per pass.  Counts are not zeroed by the launches.
struct BatchArgs {
    const uint32_t *fn = nullptr;          // ids of the batch's functions
    uint32_t nfun = 0;
    const uint64_t *tt_off = nullptr;      // byte offset of the ON table in arena
    const uint64_t *dc_off = nullptr;      // byte offset of the DC table, ~0: none
    const uint64_t *bm_off = nullptr;      // byte offset of the bitmap in bitmaps
    const uint8_t *arena = nullptr;
    uint8_t *bitmaps = nullptr;
    unsigned long long *count = nullptr;   // one per function id
    void *scratch = nullptr;               // n = 14 in one CTA: 3^8 * 32 bytes per CTA slot
    uint32_t scratch_ctas = 0;
};

// Enqueue the whole sweep.  d_count must point to a uint64 (zeroed here).
// Passes [first, last) only (0 .. passes.size() for the whole sweep); pass 0
// zeroes *d_count first.  With a batch (n <= 12), one CTA per function and
// d_on / d_dc / d_bitmap / d_count are unused.  tt_invert = ~0u sweeps the
// complement: the support is (not ON) or DC instead of ON or DC.
cudaError_t launch_sweep(const Plan &plan, const void *d_on, const void *d_dc,
                         void *d_state, uint32_t *d_bitmap, unsigned long long *d_count,
                         cudaStream_t stream, int first = 0, int last = -1,
                         const BatchArgs *batch = nullptr, uint32_t tt_invert = 0);

// Bytes pass i moves by design (rows read and written x 32, truth tables, bitmap).
uint64_t pass_bytes(const Plan &plan, int i, bool with_dc);

// Control block at the start of ctrl_off: uint32 error word, then ticket
// counters, then phase counters, then (8-aligned) uint64 look-back slots.
constexpr int kCtrlTickets = 8;
struct CtrlLayout {
    uint64_t err = 0;           // uint32 index
    uint64_t tickets = 1;       // uint32 index
    uint64_t done = 1 + kCtrlTickets;
    uint64_t status_u64 = 0;    // uint64 index from ctrl base
    uint64_t bytes = 0;
};
CtrlLayout ctrl_layout(const Plan &p);

// Status word written by a timed-out device wait (dqmc_dev_status reads it).
constexpr uint32_t kErrTimeout = 0x54494d45u;  // "TIME"
// Status word of the checked build when an index fell outside its buffer.
constexpr uint32_t kErrBounds = 0x424f554eu;   // "BOUN"

// Enqueue passes [first, last) of a plan (n >= 13, dqmc_pass.cu).  d_pairs
// may be null (no list).  With a batch, d_state holds one state per batch
// function (state_rows rows each), d_on / d_dc / d_bitmap / d_count / d_pairs
// are unused and no list is written.
cudaError_t launch_super(const Plan &plan, const void *d_on, const void *d_dc, void *d_state,
                         uint32_t *d_bitmap, unsigned long long *d_count, uint32_t *d_pairs,
                         uint64_t cap, void *d_ctrl, cudaStream_t stream, int first, int last,
                         const BatchArgs *batch = nullptr, uint32_t tt_invert = 0, bool inplace = false);

// Test hook: a device wait on a counter nothing sets; it must time out.
cudaError_t launch_selftest_wait(void *d_ctrl, uint64_t ctrl_bytes, uint64_t wait_ns, cudaStream_t stream);

// Whole functions in shared memory (dqmc_fn.cu), 5 <= n <= 14: tg threads
// per function, fpc functions per CTA, the high digits merged and reduced
// `digits` (2 or 3) at a time; or one function per cluster of ctas = 3
// (n = 13, 14) or 9 (n = 14) CTAs; or, for n = 14 with ctas = 1, one CTA per
// function doing the three thirds of the top digit in turn (persistent, with
// BatchArgs::scratch).
constexpr int kFnMinN = 5;
constexpr int kFnMaxN = 14;
constexpr uint64_t kFnMaxSmem = 232448;    // 227 KB of shared memory per CTA
constexpr uint64_t kFnThirdBytes = 6561ull * 32;   // one third of an n = 14 state (3^8 rows)
struct FnConfig {
    int tg = 256;
    int fpc = 1;
    int digits = 2;
    int ctas = 1;
};
uint64_t fn_smem_bytes(int n, int fpc, int ctas);
bool fn_config_ok(int n, const FnConfig &c);
// Counts are not zeroed; bitmaps and counts come from the batch tables.
cudaError_t launch_fn_batch(int n, const BatchArgs &b, const FnConfig &c, cudaStream_t s);

// The batch in one persistent launch (dqmc_fn.cu): one CTA of kQueueThreads
// threads per SM; the functions of each n wait in a queue of their own (ids
// b.fn[first .. first + count)), the queues largest n first.  A CTA takes the
// queues in turn, split into `groups` thread groups of tg threads for that n;
// a group takes one function at a time from the queue's counter (ctr[class],
// zeroed before the launch).  n <= 4: one warp per function; 5 <= n <= 13:
// the whole function in shared memory, `digits` high digits per step;
// n = 14: the whole CTA, the thirds of the top digit in turn with the CTA's
// scratch slot (b.scratch, at least `ctas` slots).
constexpr int kQueueThreads = 1024;
struct QueueClass {
    uint32_t n = 0, first = 0, count = 0;
    uint32_t tg = 32, groups = 1, digits = 3;
};
struct QueueSetup {
    uint32_t nclass = 0;
    QueueClass cls[kFnMaxN + 1];
    uint32_t *ctr = nullptr;
    uint32_t ctas = 0;
    uint64_t smem = 0;          // dynamic shared memory of the launch
};
uint64_t queue_fn_smem(int n);  // shared memory one function of n takes in the queue kernel
cudaError_t launch_fn_queue(const BatchArgs &b, const QueueSetup &q, cudaStream_t s);

// Sweep a batch of functions of one n <= 14 without device state: the
// shared-memory kernel with the batch table's shape for n (the built-in
// shared-memory shape if the table says the tile path), the one-tile kernel
// below n = 5.
cudaError_t launch_batch_in_smem(int n, const BatchArgs &b, cudaStream_t s);

// Enqueue compaction of a dense bitmap into (mask, value) pairs.
constexpr int kListWordsPerBlock = 4096;
cudaError_t launch_compact(int n, const uint32_t *d_bitmap, uint32_t *d_pairs, uint64_t cap,
                           unsigned long long *d_count, uint32_t *d_blk_counts,
                           unsigned long long *d_blk_offs, cudaStream_t stream);

}  // namespace dqmc
