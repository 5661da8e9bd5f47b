// stage_fp32.cuh -- the FP32 fused RK stage of the split ideal-MHD system
// (section 2 of arXiv 1710.06423), built for B300 (sm_103a).
//
// Data layout ("field pairs"): the six conserved perturbations are stored as
// three float2 planes P0 = (rho~, e~), P1 = (m_x, m_y), P2 = (B~x, B~y) (and
// the background as (rho_b, e_b), (B_bx, B_by)).  Every variable gets the same
// hyper-diffusion arithmetic and the flux of each pair has a common form, so
// one packed f32x2 instruction (fma/add/sub/mul.rn.f32x2) advances two
// variables at once and every stencil offset stays an aligned 8-byte access.
//
// One CTA owns a TX x TY tile at a time (32 x 32 with 256 threads, two per SM,
// unless the autotuner picked another shape) and walks the tiles of the grid
// persistently:
//   0. stage the tile + 3-cell halo of the three planes into shared memory
//      (rows 16-byte aligned): one 3D tensor copy (TMA, cp.async.bulk.tensor)
//      per plane on an mbarrier in the persistent kernel; bulk row copies in
//      the batch kernel's persistent mode, 16-byte cp.async.cg otherwise;
//   1. per staged cell: v = m/rho, total pressure, energy-flux factor, B.v,
//      the x fluxes (cells x0-2..x0+TX+1 of the tile rows) and y fluxes
//      (rows y0-2..y0+TY+1 of the tile columns) of all three pairs;
//   2. shock indicator s = max(0, -div v) around the tile;
//   3. X sweep: each thread walks SEG = 4 cells of one row with register
//      windows: face differences d1, d3, the max over three faces, the face
//      hyper-diffusion flux and the x flux derivative -> k_x (kept in shared
//      memory over the dead x-flux buffer);
//   4. Y sweep: each thread walks 4 cells of one column the same way, adds
//      k_x, applies the RK stage update (D scheme, see below), stores the
//      stage output and, in stage 4, folds the signal speed of the new state
//      into a per-thread maximum (reduced once per CTA).  Its plane loop
//      issues the next tile's staging plane by plane.
// The RK registers U0/D of a thread's Y-sweep cells are prefetched into L2
// when the tile starts and loaded into registers ahead of their use.
// A small kernel after each stage fills the ghost frame of the output
// (periodic/outflow copies), so the tile code has no boundary cases; in the
// tile configurations with in-kernel ghosts the stage kernel writes that frame
// itself after each tile near a side (tile_ghosts).
//
// RK registers (D scheme, 22.5 values moved per cell-stage):
//   s1: S1 = U0 + dt/2 k1
//   s2: D = (S1 - U0)/3 + dt/3 k2,  S2 = U0 + dt/2 k2
//   s3: D += dt/3 k3,               S3 = U0 + dt k3
//   s4: U0 = U0 + (D + dt/6 k4)
// (S1 - U0 is exact when both are within a factor of two, so the new state is
// rounded once per step.)
#pragma once
#include <cuda.h>
#include "sac_internal.cuh"
#include "speed.cuh"

namespace sac {
namespace f32k {

// ---- packed f32x2 arithmetic ------------------------------------------------
__device__ __forceinline__ float2 add2(float2 a, float2 b)
{
    float2 r;
    asm("{.reg .b64 A, B, D; mov.b64 A, {%2, %3}; mov.b64 B, {%4, %5};"
        " add.rn.f32x2 D, A, B; mov.b64 {%0, %1}, D;}"
        : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}
__device__ __forceinline__ float2 sub2(float2 a, float2 b)
{
    float2 r;
    asm("{.reg .b64 A, B, D; mov.b64 A, {%2, %3}; mov.b64 B, {%4, %5};"
        " sub.rn.f32x2 D, A, B; mov.b64 {%0, %1}, D;}"
        : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b)
{
    float2 r;
    asm("{.reg .b64 A, B, D; mov.b64 A, {%2, %3}; mov.b64 B, {%4, %5};"
        " mul.rn.f32x2 D, A, B; mov.b64 {%0, %1}, D;}"
        : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c)
{
    float2 r;
    asm("{.reg .b64 A, B, C, D; mov.b64 A, {%2, %3}; mov.b64 B, {%4, %5}; mov.b64 C, {%6, %7};"
        " fma.rn.f32x2 D, A, B, C; mov.b64 {%0, %1}, D;}"
        : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return r;
}
__device__ __forceinline__ float2 splat(float v) { return make_float2(v, v); }
__device__ __forceinline__ float max3(float a, float b, float c)
{
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}
__device__ __forceinline__ float rcp_approx(float v)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}

// Bring the 256 bytes at p (inside an allocation) into L2: three per-thread
// line prefetches.  (A bulk prefetch takes a uniform operand, so lanes with
// different addresses would be issued one after another.)
__device__ __forceinline__ void prefetch_l2_256(const void* p)
{
    const char* c = reinterpret_cast<const char*>(p);
    asm volatile("prefetch.global.L2 [%0];" :: "l"(c));
    asm volatile("prefetch.global.L2 [%0];" :: "l"(c + 128));
    asm volatile("prefetch.global.L2 [%0];" :: "l"(c + 255));
}
// 16-byte copy through L2 only (no L1 allocation); predicated without a
// branch: no copy and no read of gmem when pred is false
__device__ __forceinline__ void cp_async16_cg_if(unsigned sdst, const void* gmem, bool pred)
{
    asm volatile("{\n .reg .pred q;\n setp.ne.b32 q, %2, 0;\n @q cp.async.cg.shared.global [%0], [%1], 16;\n}"
                 :: "r"(sdst), "l"(gmem), "r"((int)pred) : "memory");
}
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity)
{
    unsigned ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Wait for the phase of *bar with the given parity; false if it has not
// completed within about one second (the copies it counts did not land).
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (!mbar_try_wait(bar, parity))
        if (global_ns() - t0 > 1000000000ull) return false;
    return true;
}
__device__ __forceinline__ void bulk_row_g2s(unsigned sdst, const void* gsrc, unsigned bytes, unsigned long long* bar)
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 :: "r"(sdst), "l"(gsrc), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;" ::: "memory");
}

// Scalar arithmetic of the element phases with every product/sum pairing
// spelled out (fma_/mul_ are the round-to-nearest intrinsics): the compiler
// may not contract them on its own, so the FP32 result depends only on this
// source, not on how the surrounding code is shaped or inlined (the single-run
// and batch kernels share the tile code and must agree bit for bit).
__device__ __forceinline__ float fma_(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ float mul_(float a, float b) { return __fmul_rn(a, b); }

// Division flavours (compile-time): the fast path uses rcp.approx for 1/rho and
// for the hyper-diffusion ratio; SAC_FP32_IEEE_DIV=1 selects correctly rounded
// division for both (accuracy studies).
#ifndef SAC_FP32_IEEE_DIV
#define SAC_FP32_IEEE_DIV 0
#endif
__device__ __forceinline__ float fdiv(float a, float b)
{
#if SAC_FP32_IEEE_DIV
    return __fdiv_rn(a, b);
#else
    return mul_(a, rcp_approx(b));
#endif
}

// ---- tile geometry ------------------------------------------------------------
// A tile is TX x TY cells (TX a multiple of the warp width, TY of the segment
// length); one CTA of NT = TX * TY / SEG threads owns it.  X sweep: thread =
// (row tid % TY, SEG-cell segment tid / TY); Y sweep: thread = (column
// tid % TX, SEG-cell segment tid / TX): one segment per thread in both.
// The autotuner chooses among the shapes instantiated below (32 x 32, 64 x 16,
// 32 x 16); every shape gives bit-for-bit the same results, since each cell's
// arithmetic does not depend on where the tile boundaries fall.
constexpr int SEG = 4;
template <int TX_, int TY_>
struct Geo {
    static constexpr int TX = TX_, TY = TY_, NT = TX * TY / SEG, NW = NT / 32;
    // staged region (cols x0-4.., rows y0-3..); its rows start 16-byte aligned
    // (pitch RXP float2) so that TMA or 16-byte cp.async.cg copies can fill it.
    // The price is a 2-way bank conflict in the X sweep's column-wise window
    // loads; measured 8% faster overall than an odd (conflict-free) pitch
    // filled by 8-byte cp.async, and the bulk copies another 2%.
    static constexpr int RX = TX + 8, RY = TY + 6, RXP = RX + 2;
    static constexpr int VXP = RX + 1;                      // row pitch of the velocity arrays (odd)
    static constexpr int FXW = TX + 4, FXP = FXW + 1;       // x fluxes: cols x0-2 .. x0+TX+1
    static constexpr int FYH = TY + 4, FYP = TX + 1;        // y fluxes: rows y0-2 .. y0+TY+1 (odd pitch)
    static constexpr int SW = TX + 2, SH = TY + 2, SP = SW + 1;   // shock indicator: x0-1.., y0-1..
    static constexpr int KXP = TX + 1;                      // k_x rows (aliases the x fluxes)
    static constexpr int PW = RX - 2;                       // primitive columns 1 .. RX-2
    // resident CTAs per SM the launch bounds ask for (128 registers a thread at
    // 256 threads; the 128-thread shape is held to three by its shared memory)
    static constexpr int MINB = NT <= 128 ? 3 : (NT <= 256 ? 2 : 1);
    static_assert(TX % 32 == 0 && TY % SEG == 0 && NT % 32 == 0, "tile shape");
    static_assert(TX <= TILE_X_MAX && TY <= TILE_Y_MAX, "the padded layout must hold a ragged last tile");
    static_assert((TY + 8) % 8 == 0, "tensor-copy destinations 128-byte aligned");
};
using G32x32 = Geo<32, 32>;
using G64x16 = Geo<64, 16>;
using G32x16 = Geo<32, 16>;

// The flux of the third pair has an exactly zero component in each direction,
// (0, F_By) along x and (F_Bx, 0) along y: only the nonzero one is stored.
template <class G>
struct Smem {
    float2 u[3][G::RY + 2][G::RXP];   // two spare rows: planes start 128-byte aligned
    union {
        struct {
            float2 fx[2][G::TY][G::FXP];   // x fluxes of pairs 0, 1
            float fx2[G::TY][G::FXP];      // F_By along x
        };
        float2 kx[3][G::TY][G::KXP];       // k_x, after the X sweep
    };
    float2 fy[2][G::FYH][G::FYP];          // y fluxes of pairs 0, 1
    float fy2[G::FYH][G::FYP];             // F_Bx along y
    float s[G::SH][G::SP];                 // shock indicator
    float vx[G::RY][G::VXP];
    float vy[G::RY][G::VXP];
    float2 ax[3], ay[3];                   // per-pair hyper-diffusion coefficients c2 cmax / d
};

// ---- ghost frame of a stage output ----------------------------------------------
// Periodic and outflow boundaries: ghost cell (gx, gy) (either coordinate
// outside the interior, up to GY cells out) holds interior cell
// (map(gx), map(gy)) in all three planes, map = wrap (periodic) or clamp to
// the edge (outflow); a ghost outside a fixed boundary keeps its value.
// Ghost t of the frame: t < GY*fw bottom rows, < 2*GY*fw top rows, then the
// left/right GY cells of each interior row (fw = nx + 2 GY).
__host__ __device__ inline long long halo_count(const Layout& L)
{
    return (long long)(L.nx + 2 * GY) * (L.ny + 2 * GY) - (long long)L.nx * L.ny;
}
__device__ __forceinline__ int halo_map(int g, int n, int bc)
{
    if (bc == BC_PERIODIC) { const int r = g % n; return r < 0 ? r + n : r; }
    return g < 0 ? 0 : n - 1;
}
__device__ __forceinline__ void halo_cell(float2* __restrict__ w, const Layout& L, int bc_x, int bc_y, long long t)
{
    const int fw = L.nx + 2 * GY;
    const long long band = (long long)GY * fw;
    int gx, gy;
    if (t < 2 * band) {
        const long long u = t < band ? t : t - band;
        const int r = (int)(u / fw);
        gx = (int)(u - (long long)r * fw) - GY;
        gy = t < band ? r - GY : L.ny + r;
    } else {
        const long long u = t - 2 * band;
        gy = (int)(u / (2 * GY));
        const int c = (int)(u - (long long)gy * (2 * GY));
        gx = c < GY ? c - GY : L.nx + (c - GY);
    }
    const bool ox = gx < 0 || gx >= L.nx, oy = gy < 0 || gy >= L.ny;
    if ((ox && bc_x == BC_FIXED) || (oy && bc_y == BC_FIXED)) return;
    const int sx = ox ? halo_map(gx, L.nx, bc_x) : gx, sy = oy ? halo_map(gy, L.ny, bc_y) : gy;
    const long long src = L.at(sx, sy), dst = L.at(gx, gy);
#pragma unroll
    for (int p = 0; p < 3; ++p) w[p * L.fstride + dst] = w[p * L.fstride + src];
}

// The same ghost frame written by the stage kernel itself (tile
// configurations with in-kernel ghosts, KG): after a tile, each thread copies
// its own Y-sweep cells (column x0 + tid % TX, rows y0 + SEG (tid / TX) + q),
// which it has just stored into w, to every ghost cell whose
// (map(gx), map(gy)) is that cell.  Along one direction the coordinates that
// hold interior coordinate i are the candidates k = 0 .. 2 GY: k = 0 is i
// itself, k = 1..GY the ghost -k and k = GY+1..2GY the ghost n+k-GY-1, a ghost
// taken when its side is not fixed and halo_map sends it to i; the cell's
// ghosts are the products of its x and y candidates other than the cell
// itself.  No kernel of the same stage reads w, and the next stage reads it
// after this kernel has completed.
__device__ __forceinline__ int ghost_coord(int k, int i, int n)
{
    return k == 0 ? i : (k <= GY ? -k : n + (k - GY - 1));
}
// Bit k set: candidate k holds i.
__device__ __forceinline__ unsigned ghost_mask(int i, int n, int bc)
{
    unsigned m = 1u;
    if (bc == BC_FIXED) return m;
    if (bc == BC_OUTFLOW) {
        if (i == 0) m |= ((1u << GY) - 1u) << 1;              // ghosts -1 .. -GY
        if (i == n - 1) m |= ((1u << GY) - 1u) << (GY + 1);   // ghosts n .. n+GY-1
        return m;
    }
    if (n >= GY) {   // periodic: ghost -k holds n - k, ghost n + k holds k
        if (i >= n - GY) m |= 1u << (n - i);
        if (i < GY) m |= 1u << (GY + 1 + i);
        return m;
    }
    for (int k = 1; k <= 2 * GY; ++k)   // periodic with fewer than GY cells: several wraps
        if (halo_map(ghost_coord(k, i, n), n, bc) == i) m |= 1u << k;
    return m;
}
// The copies of one tile near a non-fixed side.  A separate function: the
// rarely taken path then leaves the code of the tile loop as it is.
template <class G>
__device__ __noinline__ void tile_ghosts_copy(float2* __restrict__ w, const Layout L, const int bc_x, const int bc_y,
                                              const int x0, const int y0, const bool near_x, const bool near_y)
{
    const int tid = threadIdx.x, gi = x0 + tid % G::TX, j0 = y0 + (tid / G::TX) * SEG;
    if (gi >= L.nx) return;
    const unsigned mx = near_x && (gi < GY || gi >= L.nx - GY) ? ghost_mask(gi, L.nx, bc_x) : 1u;
#pragma unroll 1
    for (int q = 0; q < SEG; ++q) {
        const int gj = j0 + q;
        if (gj >= L.ny) break;
        const unsigned my = near_y && (gj < GY || gj >= L.ny - GY) ? ghost_mask(gj, L.ny, bc_y) : 1u;
        if ((mx | my) == 1u) continue;   // no ghost holds this cell
        const long long src = L.at(gi, gj);
        const float2 v0 = w[src], v1 = w[L.fstride + src], v2 = w[2 * L.fstride + src];
        for (unsigned bx = mx; bx; bx &= bx - 1u) {
            const int kx = __ffs(bx) - 1, gx = ghost_coord(kx, gi, L.nx);
            for (unsigned by = my; by; by &= by - 1u) {
                const int ky = __ffs(by) - 1;
                if ((kx | ky) == 0) continue;
                const long long dst = L.at(gx, ghost_coord(ky, gj, L.ny));
                w[dst] = v0; w[L.fstride + dst] = v1; w[2 * L.fstride + dst] = v2;
            }
        }
    }
}
// Tile-uniform test: only tiles within GY cells of a non-fixed side copy.
template <class G>
__device__ __forceinline__ void tile_ghosts(float2* __restrict__ w, const Layout& L, int bc_x, int bc_y,
                                            const int x0, const int y0)
{
    const bool near_x = bc_x != BC_FIXED && (x0 < GY || x0 + G::TX > L.nx - GY);
    const bool near_y = bc_y != BC_FIXED && (y0 < GY || y0 + G::TY > L.ny - GY);
    if (near_x || near_y) tile_ghosts_copy<G>(w, L, bc_x, bc_y, x0, y0, near_x, near_y);
}

// The shock part of the face coefficients, bh (s_f + s_{f+1}) with
// bh = c_shk / 2, on the SEG+1 faces of a segment, from the shock indicators
// s2 of its SEG+2 cells; the same for all three pairs, so computed once.
__device__ __forceinline__ void shock_faces(const float2 (&s2)[SEG + 2], float2 bh, float2 (&bsf)[SEG + 1])
{
#pragma unroll
    for (int q = 1; q <= SEG + 1; ++q) bsf[q - 1] = mul2(bh, add2(s2[q - 1], s2[q]));
}

// Face hyper-diffusion fluxes G (already divided by d^2) on the SEG+1 faces
// around a segment of SEG cells, from the SEG+6 values u of the segment plus
// a 3-cell halo on each side, and the shock parts bsf of the face
// coefficients (shock_faces):
//   d1_f = u_{f+1} - u_f,   d3_f = (u_{f+2} - u_{f-1}) - 3 d1_f,
//   R_f  = max(|d3_{f-1}|,|d3_f|,|d3_{f+1}|) / max(|d1_{f-1}|,|d1_f|,|d1_{f+1}|)  (0 if 0/0),
//   G_f  = (a R_f + (c_shk/2)(s_f + s_{f+1})) d1_f.
// A zero denominator means d1 is zero on all three faces, so G is zero: the
// denominator is clamped to 1e-30 and the product with d1 = 0 gives that 0.
template <bool SF = false>
__device__ __forceinline__ void face_fluxes(const float2 (&u)[SEG + 6], const float2 (&bsf)[SEG + 1],
                                            float2 a, float2 (&G)[SEG + 1])
{
    const float2 m3 = splat(-3.f);
    float2 d1[SEG + 3];
    float a1x[SEG + 3], a1y[SEG + 3], a3x[SEG + 3], a3y[SEG + 3];   // |d1|, |d3| per face and lane
#pragma unroll
    for (int q = 0; q < SEG + 3; ++q) {   // face f = q - 2 relative to the first cell
        d1[q] = sub2(u[q + 2], u[q + 1]);
        const float2 d3 = fma2(m3, d1[q], sub2(u[q + 3], u[q]));
        a1x[q] = fabsf(d1[q].x); a1y[q] = fabsf(d1[q].y);
        a3x[q] = fabsf(d3.x); a3y[q] = fabsf(d3.y);
    }
#pragma unroll
    for (int q = 1; q <= SEG + 1; ++q) {
        // SF: the single-face variant takes the ratio from the face itself
        const float m1x = fmaxf(SF ? a1x[q] : max3(a1x[q - 1], a1x[q], a1x[q + 1]), 1e-30f);
        const float m1y = fmaxf(SF ? a1y[q] : max3(a1y[q - 1], a1y[q], a1y[q + 1]), 1e-30f);
        const float m3x = SF ? a3x[q] : max3(a3x[q - 1], a3x[q], a3x[q + 1]);
        const float m3y = SF ? a3y[q] : max3(a3y[q - 1], a3y[q], a3y[q + 1]);
#if SAC_FP32_IEEE_DIV
        const float2 R = make_float2(fdiv(m3x, m1x), fdiv(m3y, m1y));
#else
        // one packed product of the two components' m3 * rcp(m1) (the same roundings as two scalar ones)
        const float2 R = mul2(make_float2(m3x, m3y), make_float2(rcp_approx(m1x), rcp_approx(m1y)));
#endif
        const float2 nu = fma2(a, R, bsf[q - 1]);
        G[q - 1] = mul2(nu, d1[q]);
    }
}

// Per-step constants of one run: the RK stage weights (from the device-side
// step scalars) and, in shared memory, the per-pair hyper-diffusion
// coefficients c2 cmax / d.  Loaded once per launch by the single-run kernel,
// once per tile by the batch kernel (whose tiles belong to different runs).
struct StepConsts {
    float2 h2, dt2, d3t, d6t;
};
__device__ __forceinline__ StepConsts load_step_consts(const DevScalars* sc)
{
    StepConsts k;
    k.h2 = splat(sc->fdt[0]); k.dt2 = splat(sc->fdt[1]); k.d3t = splat(sc->fdt[2]); k.d6t = splat(sc->fdt[3]);
    return k;
}
// threads 0..2 (one pair each); visible to the CTA after its next barrier
template <class G>
__device__ __forceinline__ void store_hd_coeffs(const StageArgs<float>& a, Smem<G>& S, const int tid)
{
    if (tid < 3) {
        const float cmx = a.sc->fcmax[0], cmy = a.sc->fcmax[1];
        const int f0 = tid == 0 ? 0 : (tid == 1 ? 1 : 4), f1 = tid == 0 ? 3 : (tid == 1 ? 2 : 5);
        S.ax[tid] = make_float2(a.f_c2dx[f0] * cmx, a.f_c2dx[f1] * cmx);
        S.ay[tid] = make_float2(a.f_c2dy[f0] * cmy, a.f_c2dy[f1] * cmy);
    }
}

// Block maximum of the per-thread running signal-speed keys m[0] (x), m[1] (y)
// folded into the run's cmax_bits with one atomicMax per direction.  Every
// thread of the CTA calls it (it holds a barrier).
template <int NW>
__device__ __forceinline__ void block_speed_max(const unsigned long long (&m)[2], unsigned long long (*red)[NW],
                                                DevScalars* sc)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
#pragma unroll
    for (int d = 0; d < 2; ++d) {
        unsigned long long v = m[d];
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
            v = w > v ? w : v;
        }
        if (lane == 0) red[d][warp] = v;
    }
    __syncthreads();
    if (tid < 2) {
        unsigned long long v = 0ull;
        for (int w = 0; w < NW; ++w) v = red[tid][w] > v ? red[tid][w] : v;
        atomicMax(&sc->cmax_bits[tid], v);
    }
}

// Issue the cp.async copies of plane p of the staged region of tile (x0, y0):
// warp w copies rows w, w + NW, ...; lane l copies 16 bytes (two float2) at
// chunks l, l + 32, ... of the RX / 2 chunks of a row.  Completion:
// cp_async_wait_all.
template <class G>
__device__ __forceinline__ void stage_plane(const StageArgs<float>& a, Smem<G>& S, const int x0, const int y0, const int p)
{
    constexpr int RX = G::RX, RY = G::RY, RXP = G::RXP, NW = G::NW;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const Layout L = a.L;
    const float2* gin = reinterpret_cast<const float2*>(a.sin);
    static_assert(RX % 2 == 0 && (RXP * sizeof(float2)) % 16 == 0, "16-byte staging");
    const long long rstep = (long long)NW * L.pitch;
#pragma unroll
    for (int c0 = 0; c0 < RX / 2; c0 += 32) {
        const bool act = c0 + lane < RX / 2;
        const int l2 = act ? c0 + lane : 0;
        const unsigned sbase = (unsigned)__cvta_generic_to_shared(&S.u[p][warp][2 * l2]);
        const float2* g = gin + p * L.fstride + (long long)(y0 + warp) * L.pitch + x0 + 2 * l2;
#pragma unroll
        for (int k = 0; k < (RY + NW - 1) / NW; ++k) {
            if (k * NW + warp < RY)   // warp-uniform
                cp_async16_cg_if(sbase + (unsigned)((k * NW * RXP) * sizeof(float2)), g, act);
            g += rstep;
        }
    }
}

// Pointwise RK registers U0 (stages 2-4) and D (stages 3-4) of plane p at the
// cells e_first + q * pitch, q < SEG (zero where q >= nq: outside the grid).
template <int STAGE>
__device__ __forceinline__ void load_pointwise(const StageArgs<float>& a, const long long e, const int nq,
                                               float2 (&u0v)[SEG], float2 (&dv)[SEG])
{
    const float2* __restrict__ gu0 = reinterpret_cast<const float2*>(a.u0);
    const float2* __restrict__ gacc = reinterpret_cast<const float2*>(a.acc);
#pragma unroll
    for (int q = 0; q < SEG; ++q) {
        const bool ok = q < nq;
        u0v[q] = (STAGE >= 2 && ok) ? gu0[e + q * a.L.pitch] : make_float2(0.f, 0.f);
        dv[q] = (STAGE >= 3 && ok) ? gacc[e + q * a.L.pitch] : make_float2(0.f, 0.f);
    }
}

// Persistent kernels: plane p of the staged region of tile (x0, y0), completing
// on the CTA's mbarrier.  With a tensor map of the stage input (single-run
// kernel): one 3D tensor copy of the plane's RXP x RY box (RXP float2 per row,
// the region's own pitch; coordinates past the grid read zeros), issued by one
// thread; G::kTileBytesTM per tile.  Without one (batch kernel, whose next tile
// may belong to another run): one RX-float2 bulk copy per row (lane k of warp w
// copies row w + NW k); G::kTileBytes per tile.
template <class G>
constexpr unsigned tile_bytes() { return 3u * G::RY * G::RX * sizeof(float2); }
template <class G>
constexpr unsigned tile_bytes_tm() { return 3u * G::RY * G::RXP * sizeof(float2); }
// Where the next tile's staged region comes from: its tile origin and the
// stencil input of its run (a batch's next tile may belong to another run).
struct NextTile {
    bool has;
    int x0, y0;
    const float* sin;
    long long fstride;
    int pitch;
    const CUtensorMap* tm = nullptr;   // the stage input as a 3D tensor (pitch, rows, 3 planes)
};
__device__ __forceinline__ NextTile next_tile(const StageArgs<float>& a, bool has, int x0, int y0)
{
    return NextTile{has, x0, y0, a.sin, a.L.fstride, a.L.pitch};
}
template <class G>
__device__ __forceinline__ void stage_plane_bulk(const NextTile& n, Smem<G>& S, const int p, unsigned long long* bar)
{
    static_assert((G::RY + 2) * G::RXP * sizeof(float2) % 128 == 0, "tensor-copy destinations 128-byte aligned");
    if (n.tm) {   // one tensor copy of the plane's RY x RXP box (rows of RXP float2, as the region's pitch)
        if (threadIdx.x == 0) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
                         :: "r"(smem_u32(&S.u[p][0][0])), "l"(n.tm), "r"(n.x0), "r"(n.y0), "r"(p), "r"(smem_u32(bar)) : "memory");
        }
        return;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int r = warp + G::NW * lane;
    if (lane < (G::RY + G::NW - 1) / G::NW && r < G::RY) {
        const float2* g = reinterpret_cast<const float2*>(n.sin) + p * n.fstride + (long long)(n.y0 + r) * n.pitch + n.x0;
        bulk_row_g2s(smem_u32(&S.u[p][r][0]), g, G::RX * sizeof(float2), bar);
    }
}

// One tile (x0, y0) of one run; every thread of the CTA calls it (it holds
// barriers).  OVERLAP: the caller has issued the bulk copies of this tile's
// staged region on *bar (expected at parity *phase), and the Y sweep issues
// those of the next tile (nt, if nt.has) plane by plane as soon as the CTA
// has read the plane it replaces.  The wait is bounded: if the copies do not
// land, the run's status becomes ST_ERR_TIMEOUT, *failed is set and every
// thread returns.  S.ax/S.ay must hold the run's coefficients (store_hd_coeffs).
// Stage 4 folds the signal speeds of the tile's new state into m.
template <class G, int STAGE, bool BG, bool HD, bool OVERLAP, bool GRAV = false, bool SF = false>
__device__ __forceinline__ void tile_body(const StageArgs<float>& a, const int x0, const int y0, Smem<G>& S,
                                          const StepConsts& K, unsigned long long (&m)[2],
                                          const NextTile& nt = NextTile{},
                                          unsigned long long* bar = nullptr, unsigned* phase = nullptr,
                                          bool* failed = nullptr)
{
    constexpr int TX = G::TX, TY = G::TY, NT = G::NT, NW = G::NW, RY = G::RY, FXW = G::FXW, FYH = G::FYH;
    constexpr int KXP = G::KXP, PW = G::PW, SW = G::SW, SH = G::SH;
    const Layout L = a.L;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const float2* __restrict__ gbg = reinterpret_cast<const float2*>(a.bg);
    const long long P = L.fstride;              // plane stride in float2 elements
    // region (r, c) <-> interior (x0 - 4 + c, y0 - 3 + r) <-> padded element (y0 + r) * pitch + x0 + c
    const long long rbase = (long long)y0 * L.pitch + x0;

    // this thread's cells in the Y sweep and RK update: column x0 + col, rows
    // y0 + y_0 + q (q < nq inside the grid; ragged last tiles)
    const int col = tid % TX, y_0 = (tid / TX) * SEG, gi = x0 + col;
    const long long e_first = L.at(gi, y0 + y_0);
    const int nq = gi < L.nx ? L.ny - (y0 + y_0) : 0;
    // The pointwise RK registers U0/D of these cells are brought into L2 when the
    // tile starts (one prefetch per 256-byte row segment: lane l of the warp
    // takes pair l/8, array U0 or D by (l/4)%2, row l%4 of the warp's 4 x 32
    // cells; rows inside the grid), so the register loads later in the tile hit
    // L2.  Prefetching a whole tile ahead measured slower.
    if (STAGE >= 2 && lane < 24) {
        const int pp = lane >> 3, arr = (lane >> 2) & 1, qq = lane & 3;
        if ((STAGE >= 3 || arr == 0) && y0 + y_0 + qq < L.ny)
            prefetch_l2_256(reinterpret_cast<const float2*>(arr ? a.acc : a.u0) + pp * P
                                + L.at(x0 + (col - lane), y0 + y_0 + qq));
    }

    // ---- 0. the staged region of the three planes in shared memory -----------------
    if (!OVERLAP) {
#pragma unroll
        for (int p = 0; p < 3; ++p) stage_plane(a, S, x0, y0, p);
    }
    if (OVERLAP) {
        const bool to = !mbar_wait_bounded(bar, *phase);
        if (__syncthreads_or(to)) {
            if (threadIdx.x == 0) a.sc->status = ST_ERR_TIMEOUT;
            *failed = true;
            return;
        }
        *phase ^= 1u;
    } else {
        cp_async_wait_all();
        __syncthreads();
    }

    const float gm1 = a.f_gm1;

    // ---- 1. primitives and fluxes on the staged box [x0-3, x0+TX+3) x [y0-3, y0+TY+3)
    {
        // region cell (r, c); fx_ok / fy_ok: the cell's x / y fluxes are needed
        auto prim_cell = [&](const int r, const int c, const bool fx_ok, const bool fy_ok) {
            const float2 P0 = S.u[0][r][c], P1 = S.u[1][r][c], P2 = S.u[2][r][c];
            const float mx = P1.x, my = P1.y, btx = P2.x, bty = P2.y, et = P0.y;
            float ux, uy, pt, etot, bx, by;
            float2 bb2 = make_float2(0.f, 0.f);
            if constexpr (BG) {
                const long long e = rbase + (long long)r * L.pitch + c;
                const float2 B0 = __ldg(gbg + e), B1 = __ldg(gbg + P + e);   // (rho_b, e_b), (B_bx, B_by)
                bb2 = B1;
                const float rinv = fdiv(1.f, B0.x + P0.x);
                ux = mul_(mx, rinv); uy = mul_(my, rinv);
                const float ekin = mul_(0.5f, fma_(mx, ux, mul_(my, uy)));
                const float bb = fma_(B1.x, btx, mul_(B1.y, bty));
                const float b2p = mul_(0.5f, fma_(btx, btx, mul_(bty, bty)));
                const float pk = mul_(gm1, ((et - ekin) - bb) - b2p);
                pt = (pk + bb) + b2p;
                const float b2b = mul_(0.5f, fma_(B1.x, B1.x, mul_(B1.y, B1.y)));
                const float ptb = fma_(gm1, B0.y - b2b, b2b);
                etot = ((et + B0.y) + pt) + ptb;
                bx = B1.x + btx; by = B1.y + bty;
            } else {
#if SAC_FP32_IEEE_DIV
                ux = __fdiv_rn(mx, P0.x); uy = __fdiv_rn(my, P0.x);
#else
                const float rinv = rcp_approx(P0.x);
                ux = mul_(mx, rinv); uy = mul_(my, rinv);
#endif
                const float ekin = mul_(0.5f, fma_(mx, ux, mul_(my, uy)));
                const float b2p = mul_(0.5f, fma_(btx, btx, mul_(bty, bty)));
                pt = fma_(gm1, (et - ekin) - b2p, b2p);
                etot = et + pt;
                bx = btx; by = bty;
            }
            S.vx[r][c] = ux; S.vy[r][c] = uy;
            const float bv = fma_(bx, ux, mul_(by, uy));
            // both flux sets for every cell (straight-line code); only the stores are conditional
            // x fluxes: (m_x, F_e), (F_mx, F_my), (0, F_By)
            float2 f1x = fma2(splat(ux), P1, make_float2(pt, 0.f));
            f1x = fma2(splat(-btx), P2, f1x);
            if constexpr (BG) { f1x = fma2(splat(-btx), bb2, f1x); f1x = fma2(splat(-bb2.x), P2, f1x); }
            const float2 f0x = make_float2(mx, fma_(ux, etot, -mul_(bx, bv)));
            const float2 f2x = make_float2(0.f, fma_(ux, by, -mul_(bx, uy)));
            // y fluxes: (m_y, F_e), (F_mx, F_my), (F_Bx, 0)
            float2 f1y = fma2(splat(uy), P1, make_float2(0.f, pt));
            f1y = fma2(splat(-bty), P2, f1y);
            if constexpr (BG) { f1y = fma2(splat(-bty), bb2, f1y); f1y = fma2(splat(-bb2.y), P2, f1y); }
            const float2 f0y = make_float2(my, fma_(uy, etot, -mul_(by, bv)));
            const float2 f2y = make_float2(fma_(uy, bx, -mul_(by, ux)), 0.f);
            if (fx_ok) { S.fx[0][r - 3][c - 2] = f0x; S.fx[1][r - 3][c - 2] = f1x; S.fx2[r - 3][c - 2] = f2x.y; }
            if (fy_ok) { S.fy[0][r - 1][c - 4] = f0y; S.fy[1][r - 1][c - 4] = f1y; S.fy2[r - 1][c - 4] = f2y.x; }
        };
        auto flux_ok = [](const int r, const int c, bool& fx_ok, bool& fy_ok) {
            fx_ok = (unsigned)(r - 3) < (unsigned)TY && (unsigned)(c - 2) < (unsigned)FXW;
            fy_ok = (unsigned)(r - 1) < (unsigned)FYH && (unsigned)(c - 4) < (unsigned)TX;
        };
        // Main pass: warp w, lane l -> columns 1 + l, 33 + l, ... (TX / 32 of them)
        // of rows w, w + NW, ... (one row per warp-instruction: conflict-free);
        // tail: the last PW - TX columns walked down the rows, one cell per thread
        // (a warp covers consecutive rows of a column; the odd pitches keep that
        // conflict-free).
        constexpr int NTAIL = (PW - TX) * RY;
        static_assert(PW > TX, "primitive-phase mapping");
#pragma unroll 1
        for (int k = 0; k < (RY + NW - 1) / NW; ++k) {
            const int r = warp + NW * k;
            if (r < RY) {
#pragma unroll
                for (int c0 = 0; c0 < TX; c0 += 32) {
                    bool fx_ok, fy_ok;
                    flux_ok(r, 1 + c0 + lane, fx_ok, fy_ok);
                    prim_cell(r, 1 + c0 + lane, fx_ok, fy_ok);
                }
            }
        }
        if constexpr (NTAIL <= NT) {
            if (tid < NTAIL) {
                const int cc = tid / RY, r = tid - cc * RY;
                bool fx_ok, fy_ok;
                flux_ok(r, TX + 1 + cc, fx_ok, fy_ok);
                prim_cell(r, TX + 1 + cc, fx_ok, fy_ok);
            }
        } else {
            for (int v = tid; v < NTAIL; v += NT) {
                const int cc = v / RY, r = v - cc * RY;
                bool fx_ok, fy_ok;
                flux_ok(r, TX + 1 + cc, fx_ok, fy_ok);
                prim_cell(r, TX + 1 + cc, fx_ok, fy_ok);
            }
        }
    }
    __syncthreads();

    const float inv12dx = a.f_inv12dx, inv12dy = a.f_inv12dy;

    // register loads of the first pair's pointwise values (from L2), issued before the shock phase
    float2 nu0[SEG], ndv[SEG];
    load_pointwise<STAGE>(a, e_first, nq, nu0, ndv);

    // ---- 2. shock indicator on [x0-1, x0+TX] x [y0-1, y0+TY] ---------------------
    if constexpr (HD) {
        auto shock_cell = [&](const int sr, const int scn) {
            const int r = sr + 2, c = scn + 3;
            const float dvx = mul_(fma_(8.f, S.vx[r][c + 1] - S.vx[r][c - 1], -(S.vx[r][c + 2] - S.vx[r][c - 2])), inv12dx);
            const float dvy = mul_(fma_(8.f, S.vy[r + 1][c] - S.vy[r - 1][c], -(S.vy[r + 2][c] - S.vy[r - 2][c])), inv12dy);
            const float sv = fmaxf(0.f, -(dvx + dvy));
            S.s[sr][scn] = sv;
        };
        // main pass: warp w, lane l -> columns l, 32 + l, ... of rows w, w + NW, ...;
        // tail: the last SW - TX columns walked down the rows, on the threads of
        // the warps with one main row less (a strided loop if they are too few)
        constexpr int STAIL = (SW - TX) * SH, S0 = (SH % NW) * 32;
#pragma unroll 2
        for (int k = 0; k < (SH + NW - 1) / NW; ++k)
            if (warp + NW * k < SH) {
#pragma unroll
                for (int c0 = 0; c0 < TX; c0 += 32) shock_cell(warp + NW * k, c0 + lane);
            }
        if constexpr (S0 + STAIL <= NT) {
            if (tid >= S0 && tid < S0 + STAIL) {
                const int t = tid - S0, cc = t / SH;
                shock_cell(t - cc * SH, TX + cc);
            }
        } else {
            for (int t = tid; t < STAIL; t += NT) {
                const int cc = t / SH;
                shock_cell(t - cc * SH, TX + cc);
            }
        }
        __syncthreads();
    }

    const float2 bh = splat(a.f_bh);
    const float2 m12x = splat(-inv12dx), m12y = splat(-inv12dy), eight = splat(8.f);

    // ... and of the second pair, issued before the X sweep
    float2 mu0[SEG], mdv[SEG];
    load_pointwise<STAGE>(a, P + e_first, nq, mu0, mdv);

    // ---- 3. X sweep: thread = (row lane, SEG-cell segment per warp) ---------------
    {
        const int row = tid % TY, x_0 = (tid / TY) * SEG;
        float2 kx[3][SEG];
        float2 bsfx[SEG + 1];
        if constexpr (HD) {
            float2 s2[SEG + 2];   // cells x_0-1 .. x_0+SEG (shock col = cell + 1)
#pragma unroll
            for (int q = 0; q < SEG + 2; ++q) s2[q] = splat(S.s[row + 1][x_0 + q]);
            shock_faces(s2, bh, bsfx);
        }
#pragma unroll
        for (int p = 0; p < 3; ++p) {
            float2 u[SEG + 6];   // cells x_0-3 .. x_0+SEG+2 (region col = cell + 4)
#pragma unroll
            for (int q = 0; q < SEG + 6; ++q) u[q] = S.u[p][row + 3][x_0 + 1 + q];
            float2 hx[SEG];
            if constexpr (HD) {
                float2 Gf[SEG + 1];
                face_fluxes<SF>(u, bsfx, S.ax[p], Gf);
#pragma unroll
                for (int q = 0; q < SEG; ++q) hx[q] = sub2(Gf[q + 1], Gf[q]);
            } else {
#pragma unroll
                for (int q = 0; q < SEG; ++q) hx[q] = make_float2(0.f, 0.f);
            }
            float2 F[SEG + 4];   // cells x_0-2 .. x_0+SEG+1 (fx col = cell + 2)
#pragma unroll
            for (int q = 0; q < SEG + 4; ++q)
                F[q] = p < 2 ? S.fx[p][row][x_0 + q] : make_float2(0.f, S.fx2[row][x_0 + q]);
#pragma unroll
            for (int q = 0; q < SEG; ++q) {
                const float2 d = fma2(eight, sub2(F[q + 3], F[q + 1]), sub2(F[q], F[q + 4]));
                kx[p][q] = fma2(m12x, d, hx[q]);
            }
        }
        __syncthreads();   // every thread is done with the x fluxes
        float2 (*KX)[TY][KXP] = S.kx;
#pragma unroll
        for (int p = 0; p < 3; ++p)
#pragma unroll
            for (int q = 0; q < SEG; ++q) KX[p][row][x_0 + q] = kx[p][q];
    }
    __syncthreads();

    // ---- 4. Y sweep, RK update, stores ---------------------------------------------
    const float2 (*KX)[TY][KXP] = S.kx;
    const float2 h2 = K.h2, dt2 = K.dt2, d3t = K.d3t, d6t = K.d6t, third = splat((float)(1.0 / 3.0));
    float2* __restrict__ gout = reinterpret_cast<float2*>(a.sout);
    float2* __restrict__ gacc = reinterpret_cast<float2*>(a.acc);
    float2 outv[SEG][3];
    float rcen[SEG];   // GRAV: rt at this thread's cells (pair 0), for the momentum source
    const float gxv = a.f_grav[0], gyv = a.f_grav[1];

    float2 bsfy[SEG + 1];
    if constexpr (HD) {
        float2 s2[SEG + 2];   // rows y_0-1 .. y_0+SEG (shock row = cell row + 1)
#pragma unroll
        for (int q = 0; q < SEG + 2; ++q) s2[q] = splat(S.s[y_0 + q][col + 1]);
        shock_faces(s2, bh, bsfy);
    }
    // (those of the third pair are loaded while the second is swept)
#pragma unroll
    for (int p = 0; p < 3; ++p) {
        const long long ep = p * P + e_first;
        float2 u0v[SEG], dv[SEG];
#pragma unroll
        for (int q = 0; q < SEG; ++q) { u0v[q] = nu0[q]; dv[q] = ndv[q]; }
        if (p == 0) {
#pragma unroll
            for (int q = 0; q < SEG; ++q) { nu0[q] = mu0[q]; ndv[q] = mdv[q]; }
        }
        if (p == 1) load_pointwise<STAGE>(a, ep + P, nq, nu0, ndv);
        float2 u[SEG + 6];   // rows y_0-3 .. y_0+SEG+2 (region row = cell row + 3)
#pragma unroll
        for (int q = 0; q < SEG + 6; ++q) u[q] = S.u[p][y_0 + q][col + 4];
        if (OVERLAP) {
            __syncthreads();   // plane p of this tile is read for good
            if (nt.has) {
                if (p == 0 && threadIdx.x == 0) mbar_expect_tx(bar, nt.tm ? tile_bytes_tm<G>() : tile_bytes<G>());
                stage_plane_bulk(nt, S, p, bar);
            }
        }
        float2 hy[SEG];
        if constexpr (HD) {
            float2 Gf[SEG + 1];
            face_fluxes<SF>(u, bsfy, S.ay[p], Gf);
#pragma unroll
            for (int q = 0; q < SEG; ++q) hy[q] = sub2(Gf[q + 1], Gf[q]);
        } else {
#pragma unroll
            for (int q = 0; q < SEG; ++q) hy[q] = make_float2(0.f, 0.f);
        }
        float2 F[SEG + 4];   // rows y_0-2 .. y_0+SEG+1 (fy row = cell row + 2)
#pragma unroll
        for (int q = 0; q < SEG + 4; ++q)
            F[q] = p < 2 ? S.fy[p][y_0 + q][col] : make_float2(S.fy2[y_0 + q][col], 0.f);
#pragma unroll
        for (int q = 0; q < SEG; ++q) {
            const float2 d = fma2(eight, sub2(F[q + 3], F[q + 1]), sub2(F[q], F[q + 4]));
            float2 k = add2(fma2(m12y, d, hy[q]), KX[p][y_0 + q][col]);
            const float2 ucen = u[q + 3];
            if constexpr (GRAV) {
                // gravity (section 2), after the flux and diffusion terms: m.g on e~
                // (m from pair 1, still in shared memory while pair 0 is swept) and
                // rt g on m (rt kept from pair 0)
                if (p == 0) {
                    const float2 m = S.u[1][y_0 + q + 3][col + 4];
                    k.y = __fadd_rn(k.y, fma_(m.x, gxv, mul_(m.y, gyv)));
                    rcen[q] = ucen.x;
                } else if (p == 1) {
                    k = add2(k, make_float2(mul_(rcen[q], gxv), mul_(rcen[q], gyv)));
                }
            }
            // the update is formed for every q (cells past the grid hold zero RK
            // registers); only the stores are predicated
            const long long e = ep + q * L.pitch;
            const bool in_grid = q < nq;
            float2 o;
            if (STAGE == 1) {
                o = fma2(h2, k, ucen);
            } else if (STAGE == 2) {
                const float2 dn = fma2(d3t, k, mul2(third, sub2(ucen, u0v[q])));
                if (in_grid) __stcs(gacc + e, dn);
                o = fma2(h2, k, u0v[q]);
            } else if (STAGE == 3) {
                const float2 dn = fma2(d3t, k, dv[q]);
                if (in_grid) __stcs(gacc + e, dn);
                o = fma2(dt2, k, u0v[q]);
            } else {
                o = add2(u0v[q], fma2(d6t, k, dv[q]));
            }
            if (in_grid) __stcs(gout + e, o);   // evict-first: L2 cannot keep it for the next stage
            outv[q][p] = o;
        }
    }

    if (STAGE == 4) {
#pragma unroll
        for (int q = 0; q < SEG; ++q) {
            if (q < nq) {
                float sx, sy;
                const float2 o0 = outv[q][0], o1 = outv[q][1], o2 = outv[q][2];
                if constexpr (BG) {
                    const long long e = L.at(gi, y0 + y_0 + q);
                    const float2 B0 = __ldg(gbg + e), B1 = __ldg(gbg + P + e);
                    signal_speeds<float, true>(o0.x, o1.x, o1.y, o0.y, o2.x, o2.y, B0.x, B0.y, B1.x, B1.y,
                                               a.f_gamma, sx, sy);
                } else {
                    signal_speeds<float, false>(o0.x, o1.x, o1.y, o0.y, o2.x, o2.y, 0.f, 0.f, 0.f, 0.f,
                                                a.f_gamma, sx, sy);
                }
                const unsigned long long kx_ = speed_key(sx), ky_ = speed_key(sy);
                m[0] = kx_ > m[0] ? kx_ : m[0];
                m[1] = ky_ > m[1] ? ky_ : m[1];
            }
        }
    }
}

// Persistent: each CTA walks the tiles t = blockIdx.x, blockIdx.x + gridDim.x, ...
// (row-major; the CTAs of one wave cover neighbouring tiles, so halo rows come
// from L2), copying the next tile's region into shared memory by TMA bulk
// copies while it finishes the current one.
// The step constants are read once; stage 4 keeps the signal-speed maximum of
// all its tiles in registers and reduces it once at the end.
// KG: the kernel also writes the ghost frame of its output (tile_ghosts);
// otherwise a ghost-frame kernel follows it.
template <class G, int STAGE, bool BG, bool HD, bool GRAV, bool SF = false, bool KG = false>
__global__ void __launch_bounds__(G::NT, G::MINB) stage_fp32(const StageArgs<float> a, const int ntx, const int ntiles,
                                                             const __grid_constant__ CUtensorMap tm)
{
    pdl_launch_dependents();
    pdl_wait();   // the previous kernel's output (stage input, scalars) is complete
    if (a.sc->skip || a.sc->status != ST_OK) return;   // skipped step, or an earlier stage gave up
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ unsigned long long red[2][G::NW];
    Smem<G>& S = *reinterpret_cast<Smem<G>*>(smem_raw);
    store_hd_coeffs(a, S, threadIdx.x);   // no later phase writes S.ax/S.ay
    // tensor copies need 128-byte aligned destinations; otherwise row copies
    const CUtensorMap* tmp = (smem_u32(&S.u[0][0][0]) & 127u) == 0 ? &tm : nullptr;
    const StepConsts K = load_step_consts(a.sc);
    unsigned long long m[2] = {0ull, 0ull};
    __shared__ __align__(8) unsigned long long bar;   // staging completion (one arrival + bytes per tile)
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    __syncthreads();
    unsigned phase = 0;
    bool failed = false;
    int t = blockIdx.x;
    if (t < ntiles) {
        NextTile f = next_tile(a, true, (t % ntx) * G::TX, (t / ntx) * G::TY);
        f.tm = tmp;
        if (threadIdx.x == 0) mbar_expect_tx(&bar, f.tm ? tile_bytes_tm<G>() : tile_bytes<G>());
        // (test hook: with drop_copies set no copy is issued, so the first tile's
        // bounded wait runs out and the launch reports ST_ERR_TIMEOUT)
        if (!a.sc->drop_copies) {
#pragma unroll
            for (int p = 0; p < 3; ++p) stage_plane_bulk(f, S, p, &bar);
        }
    }
    for (; t < ntiles; t += gridDim.x) {
        const int tn = t + gridDim.x;
        NextTile nt = next_tile(a, tn < ntiles, (tn % ntx) * G::TX, (tn / ntx) * G::TY);
        nt.tm = tmp;
        if constexpr (KG) {
            const int x0 = (t % ntx) * G::TX, y0 = (t / ntx) * G::TY;
            tile_body<G, STAGE, BG, HD, true, GRAV, SF>(a, x0, y0, S, K, m, nt, &bar, &phase, &failed);
            if (failed) return;
            tile_ghosts<G>(reinterpret_cast<float2*>(a.sout), a.L, a.bc_x, a.bc_y, x0, y0);
        } else {
            tile_body<G, STAGE, BG, HD, true, GRAV, SF>(a, (t % ntx) * G::TX, (t / ntx) * G::TY, S, K, m, nt, &bar,
                                                         &phase, &failed);
            if (failed) return;
        }
    }
    if (STAGE == 4) block_speed_max(m, red, a.sc);
}

}  // namespace f32k
}  // namespace sac
