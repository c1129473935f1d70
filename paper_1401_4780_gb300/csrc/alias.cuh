// alias.cuh -- row totals and the alias table on the GPU (alias.cu).
#pragma once

#include "common.cuh"

namespace asyrk {

// From p->w64 and p->b64 (filled by the row pass): p->frob2 = F (the exact sum
// of the w_i rounded once to the nearest double), p->bnorm (from the exact sum
// of the b_i^2, rounded once, then its square root), p->uniform, and, when
// the weights are not all bit-identical, the alias thresholds and rows in
// p->rec (whose thr/alias the row pass set to 2^32 - 1 / the row itself).
// Synchronises the stream.  Errors: EINVAL (F not positive and finite, or
// ||b||^2 not finite in FP64), ENOMEM, ECUDA.
int row_totals_and_alias(asyrk_problem *p, cudaStream_t s);

}  // namespace asyrk
