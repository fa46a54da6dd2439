// Kinds of the triangular solves on a vector (the wavefront solves of
// csrc/factor.cu): which triangle, and whether it is applied transposed.
#pragma once
#include "common.cuh"

namespace lsq {

// TB_UPPER_T: U^T y = c for upper U (a forward solve reading U by rows).
enum TrsvKindB { TB_LOWER = 0, TB_LOWER_T = 1, TB_UPPER = 2, TB_UNIT_LOWER = 3, TB_UPPER_T = 4 };

}  // namespace lsq
