// Host launchers of the compile-time variants of the step and batch kernels.
//
// Each kernel variant (storage type ST, GI mode, forced or not, strain-solve
// guard, isotropic density-gradient stencil) has one launcher and one
// occupancy query.  They are declared here and defined in variants.cu, which
// the build compiles once per (storage type, group of variants) so that the
// large kernels compile in parallel; dispatch.cu picks the variant of a launch
// at run time.  FP64 storage has no GUARD variants: its kernel takes the guard
// as a run-time flag.
#pragma once

#include "lbm_internal.h"

namespace lbm {

template <typename ST, int MODE, bool FORCED, bool GUARD, bool ISO>
cudaError_t step_variant_launch(const StepParams &p, const CUtensorMap &tin, const CUtensorMap &tout,
                                const void *fin, void *fout, int grid, cudaStream_t s);

// Resident blocks per SM of the variant (sets its dynamic shared-memory size).
template <typename ST, int MODE, bool FORCED, bool GUARD, bool ISO>
int step_variant_blocks();

template <typename ST, int MODE, bool FORCED>
cudaError_t batch_variant_launch(const BatchArgs &a, int grid, cudaStream_t s);

template <typename ST, int MODE, bool FORCED>
int batch_variant_blocks();

// The persistent batch kernel (packed storages, full GI kernel): steps k0 ..
// k0 + nsteps - 1 in one cooperative launch.
template <typename ST, bool FORCED>
cudaError_t batch_persistent_variant_launch(const BatchArgs &a, int k0, int nsteps, int grid, cudaStream_t s);

template <typename ST, bool FORCED>
int batch_persistent_variant_blocks();

}  // namespace lbm
