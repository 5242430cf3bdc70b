// Packed-set Lanczos driver shared by the C-ABI entry points and the serving loop.
#pragma once

#include <vector>

#include "internal.h"

namespace ftlm {

// One packed set taking part in a Lanczos launch: sector, packed set, its K
// blocks and their block ids (Philox key word 1), and an optional step limit.
struct LzSetIn {
    const ftlm_sector *sec;
    const PackedSet *ps;
    const ftlm_basis *const *blocks;
    const uint64_t *block_ids;
    int n_steps = 0;  // this set's step limit (0: the launch's n_steps; never above it)
};

// R chains on every block of every set, n_steps steps (Section 2.2).  alpha,
// beta: host [n_sets][K][R][n_steps]; steps_done: host [n_sets][K][R].  All
// sets share the group, spin, block shape and irreps.  esize: bytes of a stored
// vector element, sizeof(VT) or 2 (FP16 storage, VT = float).
template <typename VT>
ftlm_status lanczos_packed(const std::vector<LzSetIn> &sets, int R, int n_steps, uint64_t seed, int rng,
                           cudaStream_t stream, double *alpha, double *beta, int *steps_done, int esize);

}  // namespace ftlm
