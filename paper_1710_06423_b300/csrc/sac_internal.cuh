// sac_internal.cuh -- device data layout, per-context scalars and kernel
// arguments shared by the kernel translation units and the host engine.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace sac {

constexpr int NF = 6;   // conserved perturbation fields: rho~, m_x, m_y, e~, B~x, B~y
constexpr int NBG = 4;  // background fields: rho_b, e_b, B_bx, B_by
constexpr int GY = 3;   // ghost rows below/above the interior
constexpr int GX = 4;   // padded columns left of the interior (3 ghosts + 1 alignment pad)
constexpr int TILE_X_MAX = 64;   // largest tile any kernel uses (sizes the padding)
constexpr int TILE_Y_MAX = 32;

enum { BC_PERIODIC = 0, BC_FIXED = 1, BC_OUTFLOW = 2 };
enum { ST_OK = 0, ST_ERR_NONFINITE = -5, ST_ERR_TIMEOUT = -6 };

// Ghost-padded field-major layout: interior cell (i, j) of field f sits at
//   f * fstride + (j + GY) * pitch + (i + GX).
// pitch is a multiple of 32 elements (128 B for FP32) so every tile row
// starts 16-byte aligned; rows and pitch leave room for the largest tile so
// a ragged last tile reads only inside its own field.
struct Layout {
    int nx, ny;
    int pitch;          // elements per padded row
    int rows;           // padded rows per field
    long long fstride;  // elements per field
    __host__ __device__ long long at(int i, int j) const {
        return (long long)(j + GY) * pitch + (i + GX);
    }
};

// Device-resident step scalars of one run.  Written only by the step-control
// kernels (begin_step, control) and read by the stage kernels, so a whole RK
// step, or many, can be enqueued or graph-replayed without a host round trip.
struct DevScalars {
    double t;                 // time after the last started step
    double t_end;             // clip target (+inf when none)
    double dt;                // step size of the current step
    double fixed_dt;          // > 0: use this instead of the CFL step
    double cmax_step[2];      // signal speeds the current step's diffusion uses
    unsigned long long cmax_bits[2];  // running max of the latest state (FP64 bits, or FP32 bits in the low word)
    long long steps;          // steps taken since set_state
    int skip;                 // 1: the stage kernels of this step return at once
    int done;                 // t reached t_end
    int status;               // ST_OK or an error code
    int pad;
};

template <typename T>
struct StageArgs {
    const T* sin;      // stencil input of this stage (ghost-padded)
    const T* u0;       // step-start state (pointwise reads)
    T* acc;            // RK accumulator (pointwise)
    T* sout;           // stage output (ghost-padded; ghosts written for periodic/outflow)
    const T* bg;       // static background (ghost-padded) or nullptr
    DevScalars* sc;
    Layout L;
    double dx, dy, gamma;
    double c2[NF];
    double c_shk;
    int bc_x, bc_y;
};

// ---- launchers implemented in the kernel translation units --------------
cudaError_t launch_stage_fp64(const StageArgs<double>& a, int stage, bool hd, bool bg, cudaStream_t s);
cudaError_t launch_stage_fp32(const StageArgs<float>& a, int stage, bool hd, bool bg, cudaStream_t s);
// one-time kernel attribute set-up (dynamic shared memory limits); idempotent
cudaError_t prepare_stage_fp64();
cudaError_t prepare_stage_fp32();

}  // namespace sac
