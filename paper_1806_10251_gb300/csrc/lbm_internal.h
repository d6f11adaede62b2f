// Internal types shared by the translation units of the CUDA library.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/lbm.h"

namespace lbm {

// Threads per block of the stream-collide kernel: one strip of BW columns.
constexpr int BW = 128;

// Everything one launch of the step kernel needs, passed by value.
// Physical parameters are kept in double and converted once per thread.
struct StepParams {
    int nx, ny;
    int pitch;              // row stride in elements (multiple of 32)
    long long plane;        // elements per population plane (pitch * ny)
    int perx, pery;         // periodic in x / y
    int gi_mode;            // LBM_GI_*
    int guard;              // strain-solve guard on/off
    // relaxation and preconditioning constants
    double gamma;
    double w3, w4, w5, w6, w7, w8;
    // wall velocity of each side (west, east, south, north); zero for
    // stationary walls and periodic sides
    double side_u[4][2];
    double Fx, Fy;           // uniform force
    const float *force;      // optional per-cell force: [2][ny][pitch] (fx, fy)
    const uint8_t *solid;    // optional mask [ny][pitch], 1 = solid
    unsigned long long *guard_count;  // device counter, may be null
    int *error;              // device flag: set when a bounded wait expires
    // work decomposition: items = strips x segments, each segment Ly rows
    int Ly, nstrips, nitems;
};

// The launchers below are defined per storage type (one translation unit each).
// tin is the TMA descriptor of fin (3-D: x, y, population plane).
cudaError_t launch_step_f32(const StepParams &p, const CUtensorMap &tin, const void *fin, void *fout, int grid, cudaStream_t s);
cudaError_t launch_step_f16(const StepParams &p, const CUtensorMap &tin, const void *fin, void *fout, int grid, cudaStream_t s);
cudaError_t launch_step_bf16(const StepParams &p, const CUtensorMap &tin, const void *fin, void *fout, int grid, cudaStream_t s);
cudaError_t launch_step_f64(const StepParams &p, const CUtensorMap &tin, const void *fin, void *fout, int grid, cudaStream_t s);
int blocks_per_sm_f32(int gi_mode);
int blocks_per_sm_f16(int gi_mode);
int blocks_per_sm_bf16(int gi_mode);
int blocks_per_sm_f64(int gi_mode);
// Encode the TMA descriptor of a population buffer (box: one row of all planes).
cudaError_t make_tensor_map(CUtensorMap *map, int storage, void *base, int nx, int ny, int pitch, long long plane);

// Auxiliary kernels (aux_kernels.cu)
cudaError_t launch_init_eq(const StepParams &p, int storage, const double *rho, const double *ux,
                           const double *uy, void *f, cudaStream_t s);
cudaError_t launch_fields(const StepParams &p, int storage, const void *f, double *rho, double *ux,
                          double *uy, cudaStream_t s);
cudaError_t launch_residual(const StepParams &p, int storage, const void *f, double *snap_ux,
                            double *snap_uy, double *partials, int nblocks, double *result,
                            cudaStream_t s);
int residual_blocks(const StepParams &p);
cudaError_t launch_convert(const StepParams &p, int from_storage, const void *fin, int to_storage,
                           void *fout, cudaStream_t s);
cudaError_t launch_pops_to_f64(const StepParams &p, int storage, const void *f, double *out,
                               cudaStream_t s);
cudaError_t launch_pops_from_f64(const StepParams &p, int storage, const double *in, void *f,
                                 cudaStream_t s);

size_t storage_bytes(int storage);

}  // namespace lbm
