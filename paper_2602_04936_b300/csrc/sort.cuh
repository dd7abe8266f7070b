// Radix sort and compaction primitives used by the index build.
#pragma once

#include "common.cuh"

namespace lcph {

constexpr int kSortThreads = 256;
constexpr int kSortItems = 8;
constexpr int kSortTile = kSortThreads * kSortItems;  // keys per onesweep tile
constexpr int kMaxPasses = 8;                         // 8-bit digits of a 64-bit key
// Tiles of a superblock: a sort of up to kSortSup * kSortMaxSups tiles takes
// each tile's digit offsets from the superblock sums its count pass adds up
// (no separate scan kernel); a larger one scans the per-tile counts.
constexpr int kSortSup = 32;
constexpr int kSortMaxSups = 128;

// Device scratch for sorting up to `cap` pairs (allocated stream-ordered).
struct SortWork {
    uint32_t cap = 0;
    uint32_t* hist = nullptr;        // [kMaxPasses][256] digit totals of each pass
    uint32_t* skip = nullptr;        // [kMaxPasses] 1 if the pass's digit is constant
    uint32_t* sel = nullptr;         // [kMaxPasses + 1] buffer each pass reads (device-decided)
    uint32_t* status = nullptr;      // per-tile digit counts: [256][tiles] (then offsets) when scanned,
                                     // else [tiles][256]
    uint32_t* sup = nullptr;         // [kMaxPasses][sups][256] digit counts of each superblock of tiles
    uint32_t sups = 0;               // superblocks of the largest sort (0: the scan is used)
    uint64_t* block_sums = nullptr;  // compaction: per-block (active, starts) counts
    uint32_t* total = nullptr;       // compaction result count (device)
    uint32_t* h_total = nullptr;     // pinned host mirror of total + skip flags
    int* err = nullptr;              // device status word
    void* arena = nullptr;           // one allocation holding the buffers above
};

int sort_work_alloc(SortWork& w, uint32_t cap, int* err, cudaStream_t s);
// Sizes and places the same buffers in caller-provided memory (no allocation).
size_t sort_work_bytes(uint32_t cap);
int sort_work_place(SortWork& w, uint32_t cap, int* err, void* base);
void sort_work_free(SortWork& w, cudaStream_t s);

// Stable LSD radix sort of (key, value) pairs by the low `key_bits` bits of
// the key.  Buffers 0 hold the input and receive the result (out_k / out_v
// point at them); buffers 1 are scratch.  Digits equal for every key are
// skipped on the device; the call never waits for the device.  With
// key_of_value (32-bit keys only), the result's keys are replaced by
// key_of_value[value] (values < n), written by the last pass.
int radix_sort_pairs_u64(uint64_t* k0, uint32_t* v0, uint64_t* k1, uint32_t* v1, uint32_t n,
                         int key_bits, SortWork& w, cudaStream_t s, uint64_t** out_k,
                         uint32_t** out_v);
int radix_sort_pairs_u32(uint32_t* k0, uint32_t* v0, uint32_t* k1, uint32_t* v1, uint32_t n,
                         int key_bits, SortWork& w, cudaStream_t s, uint32_t** out_k,
                         uint32_t** out_v, const uint32_t* key_of_value = nullptr);

// Tie compaction: given eq[i] (element i equals element i-1 on the compared
// prefix; eq[0] = 0), the "active" elements are those in a run of length >= 2.
// Writes, for the j-th active element in order, out_idx[j] = i and
// out_grp[j] = index of its run among the runs of length >= 2.  Returns the
// number of active elements in *h_count (blocks the host).
int tie_compact(const uint8_t* eq, uint32_t n, uint32_t* out_idx, uint32_t* out_grp,
                uint32_t* h_count, uint32_t* h_groups, SortWork& w, cudaStream_t s);
// The same without the host read: the counts stay in w.total[0] (active
// elements) and w.total[1] (groups).
int tie_compact_async(const uint8_t* eq, uint32_t n, uint32_t* out_idx, uint32_t* out_grp, SortWork& w,
                      cudaStream_t s);
// A small pinned host buffer of this thread (16 words).
uint32_t* pinned_words();

}  // namespace lcph
