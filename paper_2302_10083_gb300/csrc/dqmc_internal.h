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

struct Plan {
    int n = 0;
    int C = 0;              // chunk digits: min(n, 5)
    int H = 0;              // high digits: n - C
    uint64_t state_rows = 0;    // rows of the device state (0: the state lives in shared memory)
    std::vector<Pass> passes;
};

constexpr int kMaxSmemGroup = 7;    // 3^7 rows x 32 B = 70 KB of shared memory
constexpr int kMaxStreamGroup = 6;  // with one inner digit: 3^6 x 3 rows

Plan make_plan(int n);
std::string describe_plan(const Plan &p);

// Workspace layout (offsets in bytes from the workspace base, 256-aligned).
struct Workspace {
    uint64_t state_off = 0, state_bytes = 0;
    uint64_t count_off = 0;             // uint64 scratch counter
    uint64_t blk_counts_off = 0;        // uint32 per compaction block
    uint64_t blk_offs_off = 0;          // uint64 per compaction block
    uint64_t n_blocks = 0;
    uint64_t total = 0;
};
Workspace workspace_layout(int n);

uint64_t bitmap_words(int n);        // ceil(3^n / 32)
uint64_t bitmap_alloc_bytes(int n);  // ceil(3^n / 8) rounded up to 16

// Enqueue the whole sweep.  d_count must point to a uint64 (zeroed here).
// Passes [first, last) only (0 .. passes.size() for the whole sweep); pass 0
// zeroes *d_count first.
cudaError_t launch_sweep(const Plan &plan, const void *d_on, const void *d_dc,
                         void *d_state, uint32_t *d_bitmap, unsigned long long *d_count,
                         cudaStream_t stream, int first = 0, int last = -1);

// Bytes pass i moves by design (rows read and written x 32, truth tables, bitmap).
uint64_t pass_bytes(const Plan &plan, int i, bool with_dc);

// Enqueue compaction of a dense bitmap into (mask, value) pairs.
constexpr int kListWordsPerBlock = 4096;
cudaError_t launch_compact(int n, const uint32_t *d_bitmap, uint32_t *d_pairs, uint64_t cap,
                           unsigned long long *d_count, uint32_t *d_blk_counts,
                           unsigned long long *d_blk_offs, cudaStream_t stream);

}  // namespace dqmc
