// sac_internal.cuh -- device data layout, per-context scalars and kernel
// arguments shared by the kernel translation units and the host engine.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

namespace sac {

constexpr int NF = 6;   // conserved perturbation fields: rho~, m_x, m_y, e~, B~x, B~y
constexpr int NBG = 4;  // background fields: rho_b, e_b, B_bx, B_by
constexpr int GY = 3;   // ghost rows below/above the interior
constexpr int GX = 4;   // padded columns left of the interior (3 ghosts + 1 alignment pad)
constexpr int TILE_X_MAX = 64;   // largest tile any kernel uses (sizes the padding)
constexpr int TILE_Y_MAX = 32;

enum { BC_PERIODIC = 0, BC_FIXED = 1, BC_OUTFLOW = 2 };
enum { ST_OK = 0, ST_ERR_NONFINITE = -5, ST_ERR_TIMEOUT = -6 };
// tile shapes of the FP32 stage kernels (SAC_TILE_* of sac.h): 32 x 32 cells
// with 256 threads, 64 x 16 with 256 threads, 32 x 16 with 128 threads
enum { TILE_32x32 = 0, TILE_64x16 = 1, TILE_32x16 = 2, NTILE_SHAPES = 3 };
// single-run FP32 tile configurations: NTILE_SHAPES + s is shape s with the
// ghost frame of each stage output written by the stage kernel itself (no
// ghost-frame launch); the batch runs use the shapes only
enum { NTILE_CONFIGS = 2 * NTILE_SHAPES };

// field index -> (plane, component) of the FP32 pair layout:
// planes (rho~, e~), (m_x, m_y), (B~x, B~y); background (rho_b, e_b), (B_bx, B_by)
__host__ __device__ constexpr int pair_plane(int f) { return f == 0 || f == 3 ? 0 : (f <= 2 ? 1 : 2); }
__host__ __device__ constexpr int pair_comp(int f) { return f == 0 || f == 1 || f == 4 ? 0 : 1; }

// Ghost-padded layouts.  Interior cell (i, j) has the in-plane offset
//   at(i, j) = (j + GY) * pitch + (i + GX).
//  planar (FP64): field f is plane f, element f * fstride + at(i, j);
//  paired (FP32): the fields are three float2 planes (pair_plane/pair_comp),
//                 float index 2 * (plane * fstride + at(i, j)) + comp.
// pitch is a multiple of 32 elements so every tile row starts 16-byte
// aligned; rows and pitch leave room for the largest tile so a ragged last
// tile reads only inside its own plane.
struct Layout {
    int nx, ny;
    int pitch;          // elements (doubles or float2) per padded row
    int rows;           // padded rows per plane
    long long fstride;  // elements per plane
    int paired;         // 1: FP32 field-pair planes
    __host__ __device__ long long at(int i, int j) const {
        return (long long)(j + GY) * pitch + (i + GX);
    }
    // scalar index of field f (background field when bgfield) at (i, j)
    __host__ __device__ long long idx(int f, int i, int j, bool bgfield) const {
        if (!paired) return (long long)f * fstride + at(i, j);
        const int pl = bgfield ? (f >> 1) : pair_plane(f), cp = bgfield ? (f & 1) : pair_comp(f);
        return 2 * ((long long)pl * fstride + at(i, j)) + cp;
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
    int drop_copies;          // test hook (sac_debug_drop_copies): FP32 stages issue no staging copies
    float fdt[4];             // FP32 kernels: dt/2, dt, dt/3, dt/6 of the current step (rounded once)
    float fcmax[2];           // FP32 kernels: cmax_step rounded to float
};

// Programmatic dependent launch (kernels launched with the programmatic
// stream-serialisation attribute): launch_dependents lets the next kernel in the
// stream be scheduled while this one runs; wait blocks until the previous
// kernel has completed and its memory is visible.  A kernel calls wait before it
// reads anything an earlier kernel wrote, so the order of results is that of a
// plain stream; only the launch latency between kernels overlaps.  Both are
// no-ops for a kernel launched without the attribute.
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Launch `kernel` on stream s with the programmatic stream-serialisation
// attribute (see pdl_wait).
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args&&... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

__device__ __forceinline__ double decode_speed(unsigned long long b, int fp32)
{
    return fp32 ? (double)__uint_as_float((unsigned)b) : __longlong_as_double((long long)b);
}

// Start one RK step of one run: the CFL step dt = C min(dx/cmax_x, dy/cmax_y)
// from the signal speeds of the current state (section 2: the maximum wave
// speed sets the step and the hyper-viscosity), clipped so that t lands on
// t_end; those speeds scale the hyper-diffusion of the step's four stages.
// A non-finite speed or step marks the run failed and skips its stages.
__device__ __forceinline__ void step_begin(DevScalars* sc, double dx, double dy, double courant, int fp32,
                                           double dt_override)
{
    if (sc->status != ST_OK || sc->done) { sc->skip = 1; return; }
    double cx = decode_speed(sc->cmax_bits[0], fp32), cy = decode_speed(sc->cmax_bits[1], fp32);
    double dt;
    if (dt_override > 0.0) dt = dt_override;
    else if (sc->fixed_dt > 0.0) dt = sc->fixed_dt;
    else { double tx = dx / cx, ty = dy / cy; dt = courant * fmin(tx, ty); }
    if (!(dt > 0.0) || !isfinite(dt) || !isfinite(cx) || !isfinite(cy)) {
        sc->status = ST_ERR_NONFINITE; sc->skip = 1; return;
    }
    int last = 0;
    if (sc->t + dt >= sc->t_end) { dt = sc->t_end - sc->t; last = 1; }
    sc->dt = dt;
    sc->cmax_step[0] = cx; sc->cmax_step[1] = cy;
    sc->fdt[0] = (float)(0.5 * dt); sc->fdt[1] = (float)dt;
    sc->fdt[2] = (float)(dt / 3.0); sc->fdt[3] = (float)(dt / 6.0);
    sc->fcmax[0] = (float)cx; sc->fcmax[1] = (float)cy;
    sc->t = last ? sc->t_end : sc->t + dt;
    sc->steps += 1;
    if (last) sc->done = 1;
    sc->cmax_bits[0] = sc->cmax_bits[1] = 0ull;
    sc->skip = 0;
}

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
    int hd_single_face;   // 1: hyper-diffusion ratio from the face itself (no max over 3 faces)
    int kernel_ghosts = 0;   // FP32 single-run kernel: 1 = it writes the ghost frame of sout itself
    double grav[2];    // gravitational acceleration; sources rt g (momentum), m.g (energy)
    int tile = TILE_32x32;   // FP32 kernels: tile shape (TILE_*)
    __host__ __device__ bool has_grav() const { return grav[0] != 0.0 || grav[1] != 0.0; }
    // FP32 kernels: the parameters above rounded once on the host, so a tile
    // does no double arithmetic (FP64 issues at 1/64 of the FP32 rate here)
    float f_gm1, f_gamma, f_bh;          // gamma - 1, gamma, c_shk / 2
    float f_inv12dx, f_inv12dy;          // 1 / (12 dx), 1 / (12 dy)
    float f_c2dx[NF], f_c2dy[NF];        // c2_f / dx, c2_f / dy
    float f_grav[2];                     // grav
    __host__ void derive_f32()
    {
        f_gm1 = (float)(gamma - 1.0); f_gamma = (float)gamma; f_bh = (float)(0.5 * c_shk);
        f_inv12dx = (float)(1.0 / (12.0 * dx)); f_inv12dy = (float)(1.0 / (12.0 * dy));
        for (int f = 0; f < NF; ++f) { f_c2dx[f] = (float)(c2[f] / dx); f_c2dy[f] = (float)(c2[f] / dy); }
        f_grav[0] = (float)grav[0]; f_grav[1] = (float)grav[1];
    }
};

// ---- launchers implemented in the kernel translation units --------------
cudaError_t launch_stage_fp64(const StageArgs<double>& a, int stage, bool hd, bool bg, cudaStream_t s);
cudaError_t launch_stage_fp32(const StageArgs<float>& a, int stage, bool hd, bool bg, cudaStream_t s);
// the tensor map of a FP32 stage input (3D: pitch float2 x padded rows x 3 planes,
// box of one staged plane of the tile shape a.tile), cached per buffer, layout
// and box (kernels_fp32.cu)
cudaError_t encode_stage_tensor_map(const StageArgs<float>& a, CUtensorMap* out);
// one-time kernel attribute set-up (dynamic shared memory limits); idempotent
cudaError_t prepare_stage_fp64();
cudaError_t prepare_stage_fp32();

}  // namespace sac
