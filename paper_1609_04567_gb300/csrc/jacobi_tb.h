// jacobi_tb.h -- temporal-blocked 2D Helmholtz Jacobi (jacobi_tb.cu).
#pragma once

#include "slr_internal.cuh"

namespace slr {

// Most sweeps one pass of the temporal-blocked Jacobi loop can fuse (its tile halo).
constexpr int kJacobiTbMaxK = 8;

// Whether the temporal-blocked loop accepts p with state buffers a, b and
// right-hand side f: SLR_J2D5, binary32 arithmetic (storage F32, BF16 or F16),
// a Dirichlet ghost value exact in the storage type, rows of whole 16-byte
// groups, 16-byte aligned arrays.
bool jacobi_tb_supported(const Problem &p, const void *a, const void *b, const void *f);

// Sweeps per pass for p: 1 (the one-sweep kernels) for temporal_k 1 or a
// problem the loop does not accept; temporal_k clamped to kJacobiTbMaxK; for
// temporal_k 0, kJacobiTbMaxK when tiling is SLR_TILING_AUTO, else 1.
int jacobi_tb_resolve_k(const Problem &p, const void *a, const void *b, const void *f);

// The whole repeat-until loop with k = jacobi_tb_resolve_k(...) > 1 sweeps per
// pass, in one cooperative launch.
cudaError_t jacobi_tb_persistent(const Problem &p, LoopArgs la, cudaStream_t st);

}  // namespace slr
