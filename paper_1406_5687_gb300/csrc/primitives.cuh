// primitives.cuh -- device-wide building blocks: LSD radix sort of uint64 keys.
#pragma once

#include "common.cuh"

namespace tcg {

// Sort keys[0..n) ascending by bits [lo_bit, lo_bit + nbits) (bits above must be zero),
// with stable 8-bit LSD passes: keys equal in those bits keep their input order.  tmp: n uint64 of scratch.  *result receives whichever of
// keys / tmp holds the sorted sequence.  Scratch for the digit counts comes from `al`.
// A look-back wait that exceeds spin_limit iterations sets TC_ERR_TIMEOUT in *err (the
// caller must check it before using the result).
// counts: optional (device, ceil(nbits / 8) * 256 uint64): the digit counts of the keys,
// gathered by the kernel that wrote them (DigitCounts below); the sort then skips its own
// counting pass and uses the array as scratch.
//
// out: optional writer of one pass (pass `pass`, or the last when -1), which writes the keys
// and also, in sorted order, what the caller builds from them:
//   OS_OUT_RUNS   per run of equal field f = (key >> fshift) & fmask among the keys other than
//                 `skip`, cnt[f] += run length (cnt zeroed by the caller).  At a pass whose
//                 output is ordered by that field this costs one atomic per run of equal f;
//                 at any pass the counts are exact.
//   OS_OUT_LISTS  OS_OUT_RUNS, plus cols[g] = key & (2^b - 1) for every key.
// Fields at or above nvert are never counted (the writer never indexes past cnt).
// A pass that starts after the error word was set does nothing, so a sort that gave up never
// reorders keys it did not place; its output is then undefined and the caller must check *err
// before any kernel reads it.
// *applied tells whether the writer ran (with n <= 1 or no bits no pass runs: the caller then
// builds that output itself).
enum { OS_OUT_KEYS = 0, OS_OUT_RUNS = 1, OS_OUT_LISTS = 2 };
struct OsOut {
    int mode = OS_OUT_KEYS;
    int pass = -1;
    int fshift = 0;
    uint64_t fmask = ~0ull;
    uint64_t skip = ~0ull;
    int32_t* cnt = nullptr;
    uint32_t nvert = 0;
    int b = 0;
    int32_t* cols = nullptr;
};

tc_status radix_sort_u64(uint64_t* keys, uint64_t* tmp, int64_t n, int lo_bit, int nbits, Allocator* al,
                         cudaStream_t s, uint64_t** result, DevStatus* err, long long spin_limit,
                         unsigned long long* counts = nullptr, const OsOut* out = nullptr, bool* applied = nullptr);

// Digit counts of the keys a kernel writes, for radix_sort_u64 over bits
// [lo_bit, lo_bit + 8 npass): the block counts into npass * 256 shared counters (dynamic
// shared memory of digit_counts_bytes) and adds them to `global` (zeroed by the caller) at
// its end.  Every thread of the block calls init and flush.
struct DigitCounts {
    unsigned long long* global;
    int lo_bit;
    int npass;
};

inline size_t digit_counts_bytes(const DigitCounts& dc) { return (size_t)dc.npass * 256 * sizeof(unsigned); }

__device__ __forceinline__ void digit_counts_init(const DigitCounts& dc, unsigned* sh) {
    for (int i = threadIdx.x; i < dc.npass * 256; i += blockDim.x) sh[i] = 0u;
    __syncthreads();
}

__device__ __forceinline__ void digit_counts_add(const DigitCounts& dc, unsigned* sh, uint64_t key) {
    const uint64_t k = key >> dc.lo_bit;
    for (int p = 0; p < dc.npass; ++p) atomicAdd(&sh[p * 256 + (unsigned)((k >> (8 * p)) & 0xFF)], 1u);
}

__device__ __forceinline__ void digit_counts_flush(const DigitCounts& dc, const unsigned* sh) {
    __syncthreads();
    for (int i = threadIdx.x; i < dc.npass * 256; i += blockDim.x)
        if (sh[i]) atomicAdd(&dc.global[i], (unsigned long long)sh[i]);
}

// Bytes of scratch radix_sort_u64 takes from the allocator for n keys (for budgets).
int64_t radix_sort_scratch_bytes(int64_t n);

}  // namespace tcg
