// primitives.cuh -- device-wide building blocks: LSD radix sort of uint64 keys.
#pragma once

#include "common.cuh"

namespace tcg {

// Sort keys[0..n) ascending by their low `nbits` bits (bits above must be zero), with
// stable 8-bit LSD passes.  tmp: n uint64 of scratch.  *result receives whichever of
// keys / tmp holds the sorted sequence.  Scratch for the digit counts comes from `al`.
tc_status radix_sort_u64(uint64_t* keys, uint64_t* tmp, int64_t n, int nbits, Allocator* al,
                         cudaStream_t s, uint64_t** result);

// Bytes of scratch radix_sort_u64 takes from the allocator for n keys (for budgets).
int64_t radix_sort_scratch_bytes(int64_t n);

}  // namespace tcg
