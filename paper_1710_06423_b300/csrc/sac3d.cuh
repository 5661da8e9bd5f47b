// sac3d.cuh -- definitions shared by the two translation units of the 3D
// form: sac3d.cu (host engine, FP64 kernels and the diagnostics, compiled
// without FMA contraction so that FP64 follows the oracle's rounding order)
// and sac3d_f32.cu (the FP32 stage and shock-indicator kernels, compiled with
// contraction).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

namespace sac3d {

constexpr int NF3 = 8;   // rho, m_x, m_y, m_z, e, B_x, B_y, B_z
constexpr int G3 = 3;    // ghost width in y and z (and at least this in x)
constexpr int GX = 4;    // left ghost width in x: with ex a multiple of 4 every row
                         // segment starting at a multiple of 4 cells is 16-byte aligned

struct Grid3 {
    int nx, ny, nz;
    long long ex, ey, ez;   // ghost-extended extents: ex = round_up(nx + 8, 4), ey = ny + 6, ez = nz + 6
    long long ne;           // cells per extended field
    __host__ __device__ long long at(int i, int j, int k) const
    {
        return ((long long)(k + G3) * ey + (j + G3)) * ex + (i + GX);
    }
};

namespace f3 {
constexpr int TX = 32, TY = 4, NT = TX * TY;   // one warp per y row of the tile
constexpr int HXS = 4, RW = TX + 2 * HXS;      // staged x range i0-4 .. i0+TX+3
constexpr int RH = TY + 2 * G3;                // staged rows j0-3 .. j0+TY+2
constexpr int NS = NF3 + 1;                    // eight fields and the shock indicator
constexpr int FXW = TX + 4, FYH = TY + 4;      // flux extents: x i0-2 .. i0+TX+1, y j0-2 .. j0+TY+1
// shock-indicator kernel: 32 x 4 output columns, staged planes of (rho, m) with a 2-cell x/y halo
constexpr int STX = 32, STY = 4, SNT = STX * STY, SRW = 40, SRH = STY + 4;
constexpr int SNB = 4;   // ring of staged planes (8 measured 3% slower: fewer resident CTAs)

struct Coef {
    float a[NF3][3];   // c2_f d cmax_d
    float bsh[3];      // c_shk d^2 / 2 (the face mean of the two shock values folds in the 1/2)
    float i12[3];      // 1 / (12 d)
    float idd[3];      // 1 / d^2
    float gm1, gamma, dt, h, d6;
    int hd;
    int drop;          // test hook (sac3_debug_drop_copies): issue no copies, so the first wait runs out
    int kz;            // planes per CTA (z chunk)
};
// tensor maps of one stage launch: the stage input (4D: x, y, z, field) and the
// shock indicator (3D) as a staged plane box and as a column-tile box, U0 and
// the RK accumulator as column-tile boxes
struct Maps {
    CUtensorMap in_full, in_col, sh_full, sh_col, u0_col, acc_col;
};

// one-time kernel attribute set-up (dynamic shared memory of the stage kernel)
cudaError_t prepare();
// RK stage `stage` (1..4) of the fused FP32 kernel; out == u0 in stage 4, in == u0
// in stage 1; stage 4 also folds the signal speeds of its output into keys
cudaError_t launch_stage(int stage, const float* in, const float* sh, const float* u0, float* acc, float* out,
                         const Grid3& g, const Coef& cf, unsigned long long* keys, int* status, const Maps& m,
                         cudaStream_t st);
// shock indicator of a stage input (tensor map `tm` of its (rho, m) planes)
cudaError_t launch_shock(float* sh, const Grid3& g, const Coef& cf, int sntx, dim3 grid, int* status,
                         const CUtensorMap& tm, cudaStream_t st);
}  // namespace f3
}  // namespace sac3d
