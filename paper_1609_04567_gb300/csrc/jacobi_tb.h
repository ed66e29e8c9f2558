// jacobi_tb.h -- temporal-blocked Helmholtz Jacobi: 2D (jacobi_tb.cu) and 3D
// (jacobi_tb3.cu).
#pragma once

#include "slr_internal.cuh"

namespace slr {

// Most sweeps one pass of the temporal-blocked Jacobi loop can fuse (its tile halo).
constexpr int kJacobiTbMaxK = 8;

// Most sweeps one pass of the 3D loop fuses (its pipeline depth), and the
// library's choice for a 3D grid with temporal_k 0 and SLR_TILING_AUTO: one
// sweep per pass, which streams the 512^3 bfloat16 grid at 70% of HBM where
// the blocked loop, bound by its instruction issue, reaches about a third of
// that rate (the autotuner times k = 2 and 4 on the caller's grid).
constexpr int kJacobiTb3MaxK = 4;
constexpr int kJacobiTb3DefaultK = 1;

// Whether a temporal-blocked loop accepts p with state buffers a, b and
// right-hand side f: SLR_J2D5 or SLR_J3D7, binary32 arithmetic (storage F32,
// BF16 or F16), a Dirichlet ghost value exact in the storage type, rows of
// whole 16-byte groups, 16-byte aligned arrays.
bool jacobi_tb_supported(const Problem &p, const void *a, const void *b, const void *f);

// Sweeps per pass for p: 1 (the one-sweep kernels) for temporal_k 1 or a
// problem the loops do not accept; temporal_k clamped to the loop's most (8 in
// 2D, 4 in 3D); for temporal_k 0 with SLR_TILING_AUTO the loop's default (8 in
// 2D, kJacobiTb3DefaultK in 3D), with another tiling 1.
int jacobi_tb_resolve_k(const Problem &p, const void *a, const void *b, const void *f);

// The whole repeat-until loop with k = jacobi_tb_resolve_k(...) > 1 sweeps per
// pass, in one cooperative launch.
cudaError_t jacobi_tb_persistent(const Problem &p, LoopArgs la, cudaStream_t st);

// The ghost value is exact in p's storage type (the blocked loops keep it in
// storage form).
bool jacobi_tb_ghost_exact(const Problem &p);

// The 3D loop (jacobi_tb3.cu): its acceptance test and the launch with K
// sweeps per pass (2 <= K <= kJacobiTb3MaxK).
bool jacobi_tb3_supported(const Problem &p, const void *a, const void *b, const void *f);
cudaError_t jacobi_tb3_persistent(const Problem &p, LoopArgs la, int K, cudaStream_t st);

}  // namespace slr
