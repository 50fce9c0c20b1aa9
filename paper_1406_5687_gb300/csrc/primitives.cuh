// primitives.cuh -- device-wide building blocks: LSD radix sort of uint64 keys.
#pragma once

#include "common.cuh"

namespace tcg {

// Sort keys[0..n) ascending by bits [lo_bit, lo_bit + nbits) (bits above must be zero),
// with stable 8-bit LSD passes: keys equal in those bits keep their input order.  tmp: n uint64 of scratch.  *result receives whichever of
// keys / tmp holds the sorted sequence.  Scratch for the digit counts comes from `al`.
// A look-back wait that exceeds spin_limit iterations sets TC_ERR_TIMEOUT in *err (the
// caller must check it before using the result).
tc_status radix_sort_u64(uint64_t* keys, uint64_t* tmp, int64_t n, int lo_bit, int nbits, Allocator* al,
                         cudaStream_t s, uint64_t** result, DevStatus* err, long long spin_limit);

// Bytes of scratch radix_sort_u64 takes from the allocator for n keys (for budgets).
int64_t radix_sort_scratch_bytes(int64_t n);

}  // namespace tcg
