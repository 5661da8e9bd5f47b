// sac_ctx.h -- host-side context of one run (shared by the engine and the
// batched-run translation unit).
#pragma once
#include <cuda_runtime.h>

#include <limits>

#include "../../include/sac.h"
#include "sac_internal.cuh"

namespace sac {
constexpr int kChunk = 16;       // steps per captured multi-step graph
constexpr int kSumBlocks = 296;  // 2 x 148 SMs
}  // namespace sac

struct sac_ctx {
    sac_params p;
    sac::Layout L;
    bool fp32 = false;
    size_t esz = 8;                 // element size of the working precision
    cudaStream_t stream = nullptr;  // user stream (may be the legacy default)
    cudaStream_t cap = nullptr;     // private stream used only for graph capture
    void* u0 = nullptr;
    void* sa = nullptr;
    void* sb = nullptr;
    void* acc = nullptr;
    void* bg = nullptr;
    sac::DevScalars* sc = nullptr;
    sac::DevScalars* hsc = nullptr;      // pinned host mirror
    double* staging = nullptr;      // packed FP64 [6][ny][nx] for host transfers
    double* part = nullptr;         // [kSumBlocks][6] partial sums + [6] result
    cudaGraphExec_t g1 = nullptr;   // one CFL step
    cudaGraphExec_t gN = nullptr;   // kChunk CFL steps
    int tile = sac::TILE_32x32;     // FP32 stage kernels: tile shape (sac_set_tile / sac_tune)
    int last_stage = 0;             // stage whose output sac_halo_* act on (0: U0, the step-start state)
    double dx = 0.0, dy = 0.0;      // cell size: (x1 - x0) / nx, (y1 - y0) / ny unless sac_set_cell_size
    bool cell_override = false;
    bool have_state = false;
    double t_end_host = std::numeric_limits<double>::infinity();
    char err[512] = {0};
};


// Stage-kernel arguments of one FP32 run for RK stage 1..4 (buffer roles of
// the ping-pong registers); defined in sac_engine.cu.
void sac_fp32_stage_args(const sac_ctx* c, int stage, sac::StageArgs<float>* out);
