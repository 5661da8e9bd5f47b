// sac3d_f32.cu -- the FP32 kernels of the 3D form (section 2 of arXiv
// 1710.06423 with three-component vectors): the fused RK stage kernel and the
// shock-indicator kernel, both marching column tiles through z fed by
// tensor-map TMA copies.  This unit is compiled with FMA contraction (the FP64
// 3D kernels in sac3d.cu are not); FP32 results are checked against the FP64
// oracle within the FP32 tolerance, not bit for bit.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstddef>

#include "sac3d.cuh"

namespace sac3d {

// ---------------------------------------------------------------------------
// FP32 fused RK stage.  One CTA owns TX x TY columns and marches through kz
// planes along z.  While it works on plane k, one thread's tensor-map TMA
// copies bring plane k+1 with its x/y halo (all eight fields in one 4D box, the
// shock indicator in one 3D box), the RK registers of plane k+1 and the column
// tile of plane k+4 into shared memory (double buffer, one mbarrier per
// buffer); per plane it builds the x and y fluxes of plane k and the z flux of
// plane k+2, and then every thread forms k = H - div F for its cell and applies
// the RK register update.  Along z the face quantities |d1|, |d3|, d1 and the hyper-diffusive
// face flux roll in registers, and the z fluxes roll through a five-plane ring.
// The shock indicator comes from shock3_f32 (global, ghost-extended layout) and
// is staged beside the fields.  Arithmetic is single precision throughout
// (reciprocals, not divisions), so results differ from the FP64 order at the
// level of FP32 rounding.
namespace f3 {

struct Smem {
    float full[2][NS + 1][RH][RW];   // planes k and k+1 (one spare field-plane: 128-byte aligned buffers)
    float col[4][NS][NT];        // planes k+1 .. k+4, own column (ring by plane % 4)
    float fz[5][NF3][NT];     // z fluxes of planes k-2 .. k+2, own column (ring by plane % 5)
    float fx[NF3][TY][FXW];
    float fy[NF3][FYH][TX];
    float rk[2][2][NF3][NT];     // U0 and the RK accumulator of the own cell, planes k and k+1
    float hy[NF3][TY][TX];       // y hyper-diffusion of plane k (the y sweep of phase 1)
};


__device__ __forceinline__ float rcpf(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
constexpr unsigned kFullBytes = (unsigned)(NF3 * RH * RW * sizeof(float)), kShFullBytes = (unsigned)(RH * RW * sizeof(float));
constexpr unsigned kColBytes = (unsigned)(NS * NT * sizeof(float)), kRkBytes = (unsigned)(NF3 * NT * sizeof(float));
// every tensor-copy destination starts on a 128-byte boundary of the Smem block
static_assert(offsetof(Smem, col) % 128 == 0 && offsetof(Smem, rk) % 128 == 0, "Smem layout");
static_assert(sizeof(Smem::full[0]) % 128 == 0 && (NF3 * RH * RW * sizeof(float)) % 128 == 0, "plane buffers");
static_assert(sizeof(Smem::col[0]) % 128 == 0 && (NF3 * NT * sizeof(float)) % 128 == 0, "column ring");
static_assert(sizeof(Smem::rk[0][0]) % 128 == 0, "RK registers");
static_assert((RW * sizeof(float)) % 16 == 0 && (TX * sizeof(float)) % 16 == 0, "box rows");
__device__ __forceinline__ unsigned su32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void tma4(const void* dst, const CUtensorMap* m, int x, int y, int z, int f, unsigned long long* bar)
{
    asm volatile("cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];"
                 :: "r"(su32(dst)), "l"(m), "r"(x), "r"(y), "r"(z), "r"(f), "r"(su32(bar)) : "memory");
}
__device__ __forceinline__ void tma3(const void* dst, const CUtensorMap* m, int x, int y, int z, unsigned long long* bar)
{
    asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
                 :: "r"(su32(dst)), "l"(m), "r"(x), "r"(y), "r"(z), "r"(su32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(su32(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(su32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity)
{
    unsigned ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(ok) : "r"(su32(bar)), "r"(parity) : "memory");
    return ok != 0;
}
// wait for the phase of *bar with the given parity; false after about one second
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (!mbar_try_wait(bar, parity))
        if (global_ns() - t0 > 1000000000ull) return false;
    return true;
}

struct P3 {
    float v[3], pt, bv;
};
__device__ __forceinline__ P3 prim3(const float* u, float gm1)
{
    P3 p;
    const float ri = rcpf(u[0]);
    p.v[0] = u[1] * ri; p.v[1] = u[2] * ri; p.v[2] = u[3] * ri;
    const float ekin = 0.5f * __fmaf_rn(u[3], p.v[2], __fmaf_rn(u[2], p.v[1], u[1] * p.v[0]));
    const float b2 = 0.5f * __fmaf_rn(u[7], u[7], __fmaf_rn(u[6], u[6], u[5] * u[5]));
    p.pt = __fmaf_rn(gm1, (u[4] - ekin) - b2, b2);
    p.bv = __fmaf_rn(u[7], p.v[2], __fmaf_rn(u[6], p.v[1], u[5] * p.v[0]));
    return p;
}
// the eight fluxes along direction D
template <int D>
__device__ __forceinline__ void flux_dir(const float* u, const P3& p, float* F)
{
    const float vd = p.v[D], bd = u[5 + D];
    F[0] = u[1 + D];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const float m = __fmaf_rn(vd, u[1 + q], -(bd * u[5 + q]));
        F[1 + q] = q == D ? m + p.pt : m;
        F[5 + q] = q == D ? 0.0f : __fmaf_rn(vd, u[5 + q], -(bd * p.v[q]));
    }
    F[4] = __fmaf_rn(vd, u[4] + p.pt, -(bd * p.bv));
}
// face q lies between cells q and q+1: d1 = u[q+1] - u[q], d3 = (u[q+2] - u[q-1]) - 3 d1
__device__ __forceinline__ void face13(float um, float u0, float u1, float u2, float& d1, float& d3)
{
    d1 = u1 - u0;
    d3 = __fmaf_rn(-3.0f, d1, u2 - um);
}
// (g_right - g_left) of one direction from the seven values u[-3..3] along it
__device__ __forceinline__ float hd_line(const float* u, int s, float a, float bl, float br)
{
    const float um3 = u[-3 * s], um2 = u[-2 * s], um1 = u[-s], uc = u[0], up1 = u[s], up2 = u[2 * s], up3 = u[3 * s];
    float d1a, d3a, d1b, d3b, d1c, d3c, d1d, d3d;
    face13(um3, um2, um1, uc, d1a, d3a);   // face -2
    face13(um2, um1, uc, up1, d1b, d3b);   // face -1
    face13(um1, uc, up1, up2, d1c, d3c);   // face 0
    face13(uc, up1, up2, up3, d1d, d3d);   // face +1
    const float a1b = fabsf(d1b), a1c = fabsf(d1c), a3b = fabsf(d3b), a3c = fabsf(d3c);
    const float m1bc = fmaxf(a1b, a1c), m3bc = fmaxf(a3b, a3c);
    const float m1l = fmaxf(fabsf(d1a), m1bc), m3l = fmaxf(fabsf(d3a), m3bc);
    const float m1r = fmaxf(m1bc, fabsf(d1d)), m3r = fmaxf(m3bc, fabsf(d3d));
    const float rl = m1l > 0.0f ? m3l * rcpf(m1l) : 0.0f;
    const float rr = m1r > 0.0f ? m3r * rcpf(m1r) : 0.0f;
    return __fmaf_rn(a, rr, br) * d1c - __fmaf_rn(a, rl, bl) * d1b;
}

template <int STAGE>
__global__ void __launch_bounds__(NT, 2)
stage3_f32(const float* __restrict__ in, const float* __restrict__ sh, const float* u0, float* __restrict__ acc,
           float* out, Grid3 g, Coef cf, int ntx, unsigned long long* __restrict__ keys, int* __restrict__ status,
           const __grid_constant__ Maps tm)
// out == u0 in stage 4; in == u0 in stage 1; stage 4 also reduces the signal
// speeds of its output into keys (ordered bits of FP64 maxima, one per direction)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) unsigned long long bar[2];   // copies of planes with even / odd k
    Smem& S = *reinterpret_cast<Smem*>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int i0 = (int)(blockIdx.x % ntx) * TX, j0 = (int)(blockIdx.x / ntx) * TY;
    const int k0 = blockIdx.y * cf.kz, k1 = min(k0 + cf.kz, g.nz);
    const int x = i0 + lane, y = j0 + w;
    const bool valid = x < g.nx && y < g.ny;
    const long long P = g.ex * g.ey, ne = g.ne;
    // own column (clamped into the interior for the threads past a ragged edge)
    const long long colc = (long long)(min(y, g.ny - 1) + G3) * g.ex + (min(x, g.nx - 1) + GX);
    const auto plane = [&](int k) { return (long long)(k + G3) * P; };
    float sp_max[3] = {0.0f, 0.0f, 0.0f};
    // one thread copies plane k (8 fields + shock indicator, with halo), its RK
    // registers and the own-column tiles of planes q0 .. q1 on bar[k & 1]
    const auto issue = [&](int k, int q0, int q1) {
        if (tid == 0) {
            unsigned long long* b = &bar[k & 1];
            mbar_expect_tx(b, kFullBytes + kShFullBytes + (unsigned)(q1 - q0 + 1) * kColBytes + (STAGE != 1 ? 2u * kRkBytes : 0u));
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            if (cf.drop) return;   // test hook: the expected bytes never arrive
            tma4(&S.full[k & 1][0][0][0], &tm.in_full, i0, j0, k + G3, 0, b);        // x = i0-4, y = j0-3 (extended)
            tma3(&S.full[k & 1][NF3][0][0], &tm.sh_full, i0, j0, k + G3, b);
            for (int q = q0; q <= q1; ++q) {
                tma4(&S.col[q & 3][0][0], &tm.in_col, i0 + GX, j0 + G3, q + G3, 0, b);
                tma3(&S.col[q & 3][NF3][0], &tm.sh_col, i0 + GX, j0 + G3, q + G3, b);
            }
            if (STAGE != 1) {
                tma4(&S.rk[k & 1][0][0][0], &tm.u0_col, i0 + GX, j0 + G3, k + G3, 0, b);
                tma4(&S.rk[k & 1][1][0][0], &tm.acc_col, i0 + GX, j0 + G3, k + G3, 0, b);
            }
        }
    };
    if (*status != 0) return;   // an earlier stage of this step gave up: nothing to do
    unsigned phase = 0;   // bit b: parity of bar[b]'s next completion
    // tensor copies need 128-byte aligned destinations (all buffer offsets are multiples of 128)
    if ((su32(&S) & 127u) != 0) {
        if (tid == 0) atomicExch(status, 2);
        return;
    }
    if (tid == 0) { mbar_init(&bar[0]); mbar_init(&bar[1]); }
    __syncthreads();

    // prologue: copies of plane k0 and of the own column of planes k0+1 .. k0+3;
    // z fluxes of planes k0-2 .. k0+1; z face state of faces k0-1, k0 and the face
    // flux at k0-1/2
    issue(k0, k0 + 1, k0 + 3);
#pragma unroll 1
    for (int q = k0 - 2; q <= k0 + 1; ++q) {
        float u[NF3], F[NF3];
#pragma unroll
        for (int f = 0; f < NF3; ++f) u[f] = in[f * ne + plane(q) + colc];
        const P3 p = prim3(u, cf.gm1);
        flux_dir<2>(u, p, F);
#pragma unroll
        for (int f = 0; f < NF3; ++f) S.fz[(q + 5) % 5][f][tid] = F[f];
    }
    float zd1[NF3], za3[NF3], za1m[NF3], za3m[NF3], zg[NF3];   // face k: d1, |d3|; face k-1: |d1|, |d3|; g(k-1/2)
    if (cf.hd) {
        const float bz = cf.bsh[2] * (sh[plane(k0 - 1) + colc] + sh[plane(k0) + colc]);
#pragma unroll
        for (int f = 0; f < NF3; ++f) {
            const float* uf = in + f * ne + colc;
            float u[6];
#pragma unroll
            for (int o = 0; o < 6; ++o) u[o] = uf[plane(k0 - 3 + o)];
            float d1a, d3a, d1b, d3b, d1c, d3c;
            face13(u[0], u[1], u[2], u[3], d1a, d3a);   // face k0-2
            face13(u[1], u[2], u[3], u[4], d1b, d3b);   // face k0-1
            face13(u[2], u[3], u[4], u[5], d1c, d3c);   // face k0
            const float m1 = fmaxf(fmaxf(fabsf(d1a), fabsf(d1b)), fabsf(d1c));
            const float m3 = fmaxf(fmaxf(fabsf(d3a), fabsf(d3b)), fabsf(d3c));
            const float r = m1 > 0.0f ? m3 * rcpf(m1) : 0.0f;
            zg[f] = __fmaf_rn(cf.a[f][2], r, bz) * d1b;
            zd1[f] = d1c; za3[f] = fabsf(d3c); za1m[f] = fabsf(d1b); za3m[f] = fabsf(d3b);
        }
    }

#pragma unroll 1
    for (int k = k0; k < k1; ++k) {
        __syncthreads();   // the previous plane's readers are done
        const long long pk = plane(k);
        if (k + 1 < k1) issue(k + 1, k + 4, k + 4);   // plane k+4 <= nz + 2: inside the ghost frame
        {   // plane k's copies (bounded wait; a timeout is reported and every thread leaves)
            const int kb_ = k & 1;
            const bool to = !mbar_wait_bounded(&bar[kb_], (phase >> kb_) & 1u);
            if (__syncthreads_or(to)) {
                if (tid == 0) {
                    atomicExch(status, 1);
                    // let plane k+1's copies (if issued) land before the CTA's memory is released
                    if (k + 1 < k1 && !cf.drop) mbar_wait_bounded(&bar[kb_ ^ 1], (phase >> (kb_ ^ 1)) & 1u);
                }
                return;
            }
            phase ^= 1u << kb_;
        }
        const int kb = k & 1;

        {   // x and y fluxes of the own cell
            float u[NF3], F[NF3];
#pragma unroll
            for (int f = 0; f < NF3; ++f) u[f] = S.full[kb][f][G3 + w][HXS + lane];
            const P3 p = prim3(u, cf.gm1);
            flux_dir<0>(u, p, F);
#pragma unroll
            for (int f = 0; f < NF3; ++f) S.fx[f][w][lane + 2] = F[f];
            flux_dir<1>(u, p, F);
#pragma unroll
            for (int f = 0; f < NF3; ++f) S.fy[f][w + 2][lane] = F[f];
        }
        {   // y fluxes of the halo rows y = j0-2, j0-1, j0+TY, j0+TY+1 (one warp per row)
            const int fyr = w < 2 ? w : w + TY, sr = fyr + 1;
            float u[NF3], F[NF3];
#pragma unroll
            for (int f = 0; f < NF3; ++f) u[f] = S.full[kb][f][sr][HXS + lane];
            const P3 p = prim3(u, cf.gm1);
            flux_dir<1>(u, p, F);
#pragma unroll
            for (int f = 0; f < NF3; ++f) S.fy[f][fyr][lane] = F[f];
        }
        if (tid < 4 * TY) {   // x fluxes of the halo columns x = i0-2, i0-1, i0+TX, i0+TX+1
            const int r = tid >> 2, q = tid & 3;
            const int fxc = q < 2 ? q : q + TX, sc = fxc + 2;
            float u[NF3], F[NF3];
#pragma unroll
            for (int f = 0; f < NF3; ++f) u[f] = S.full[kb][f][G3 + r][sc];
            const P3 p = prim3(u, cf.gm1);
            flux_dir<0>(u, p, F);
#pragma unroll
            for (int f = 0; f < NF3; ++f) S.fx[f][r][fxc] = F[f];
        }
        if (cf.hd) {   // y sweep: H_y of the tile's TY rows for fields 2w, 2w+1 of column lane
            static_assert(TY == 4 && RH == 10 && NF3 == 2 * (NT / 32), "y-sweep mapping");
            const float* scol = &S.full[kb][NF3][0][HXS + lane];   // staged rows 0..RH-1 = y0-3 ..
            float bsf[TY + 1];   // shock term of the faces between rows L and L+1, L = 2 .. 6
#pragma unroll
            for (int q = 0; q <= TY; ++q) bsf[q] = cf.bsh[1] * (scol[(2 + q) * RW] + scol[(3 + q) * RW]);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int f = 2 * w + h;
                const float* ucol = &S.full[kb][f][0][HXS + lane];
                float u[RH];
#pragma unroll
                for (int i = 0; i < RH; ++i) u[i] = ucol[i * RW];
                float d1[TY + 3], a1[TY + 3], a3[TY + 3];   // faces L = 1 .. 7 (between rows L, L+1)
#pragma unroll
                for (int q = 0; q < TY + 3; ++q) {
                    float d3;
                    face13(u[q], u[q + 1], u[q + 2], u[q + 3], d1[q], d3);
                    a1[q] = fabsf(d1[q]); a3[q] = fabsf(d3);
                }
                float gy[TY + 1];   // face fluxes at faces L = 2 .. 6
#pragma unroll
                for (int q = 1; q <= TY + 1; ++q) {
                    const float m1 = fmaxf(fmaxf(a1[q - 1], a1[q]), a1[q + 1]);
                    const float m3 = fmaxf(fmaxf(a3[q - 1], a3[q]), a3[q + 1]);
                    const float r = m1 > 0.0f ? m3 * rcpf(m1) : 0.0f;
                    gy[q - 1] = __fmaf_rn(cf.a[f][1], r, bsf[q - 1]) * d1[q];
                }
#pragma unroll
                for (int r = 0; r < TY; ++r) S.hy[f][r][lane] = (gy[r + 1] - gy[r]) * cf.idd[1];
            }
        }
        {   // z flux of plane k+2, own column
            float u[NF3], F[NF3];
#pragma unroll
            for (int f = 0; f < NF3; ++f) u[f] = S.col[(k + 2) % 4][f][tid];
            const P3 p = prim3(u, cf.gm1);
            flux_dir<2>(u, p, F);
#pragma unroll
            for (int f = 0; f < NF3; ++f) S.fz[(k + 2) % 5][f][tid] = F[f];
        }
        __syncthreads();
        if (!valid) continue;

        const float* sc = &S.full[kb][NF3][G3 + w][HXS + lane];
        float bxl = 0.f, bxr = 0.f, bzr = 0.f;
        if (cf.hd) {
            bxl = cf.bsh[0] * (sc[-1] + sc[0]);
            bxr = cf.bsh[0] * (sc[0] + sc[1]);
            bzr = cf.bsh[2] * (sc[0] + S.col[(k + 1) % 4][NF3][tid]);
        }
        const int s1 = (k + 1) % 4, s2 = (k + 2) % 4, s3 = (k + 3) % 4;
        float wn[NF3];   // the stage output of the own cell
        const int zp1 = (k + 1) % 5, zm1 = (k + 4) % 5, zp2 = (k + 2) % 5, zm2 = (k + 3) % 5;
#pragma unroll
        for (int f = 0; f < NF3; ++f) {
            const float* uc = &S.full[kb][f][G3 + w][HXS + lane];
            float hsum = 0.0f;
            if (cf.hd) {
                const float hx = hd_line(uc, 1, cf.a[f][0], bxl, bxr) * cf.idd[0];
                const float hy = S.hy[f][w][lane];
                // z: the new face k+1 from planes k .. k+3, then face k+1/2
                float d1n, d3n;
                face13(uc[0], S.col[s1][f][tid], S.col[s2][f][tid], S.col[s3][f][tid], d1n, d3n);
                const float a1n = fabsf(d1n), a3n = fabsf(d3n), a1 = fabsf(zd1[f]);
                const float m1 = fmaxf(fmaxf(za1m[f], a1), a1n), m3 = fmaxf(fmaxf(za3m[f], za3[f]), a3n);
                const float r = m1 > 0.0f ? m3 * rcpf(m1) : 0.0f;
                const float gz = __fmaf_rn(cf.a[f][2], r, bzr) * zd1[f];
                const float hz = (gz - zg[f]) * cf.idd[2];
                zg[f] = gz; za1m[f] = a1; za3m[f] = za3[f]; zd1[f] = d1n; za3[f] = a3n;
                hsum = (hx + hy) + hz;
            }
            const float* fxr = &S.fx[f][w][lane + 2];
            const float* fyr = &S.fy[f][w + 2][lane];
            const float dfx = __fmaf_rn(8.0f, fxr[1] - fxr[-1], -(fxr[2] - fxr[-2])) * cf.i12[0];
            const float dfy = __fmaf_rn(8.0f, fyr[TX] - fyr[-TX], -(fyr[2 * TX] - fyr[-2 * TX])) * cf.i12[1];
            const float dfz = __fmaf_rn(8.0f, S.fz[zp1][f][tid] - S.fz[zm1][f][tid],
                                        -(S.fz[zp2][f][tid] - S.fz[zm2][f][tid])) * cf.i12[2];
            const float kf = hsum - ((dfx + dfy) + dfz);
            const long long e = f * ne + pk + colc;
            const float r0 = S.rk[kb][0][f][tid], ra = S.rk[kb][1][f][tid];
            if (STAGE == 1) {
                __stcs(&acc[e], kf);
                __stcs(&out[e], __fmaf_rn(cf.h, kf, uc[0]));
            } else if (STAGE == 2) {
                __stcs(&acc[e], __fmaf_rn(2.0f, kf, ra));
                __stcs(&out[e], __fmaf_rn(cf.h, kf, r0));
            } else if (STAGE == 3) {
                __stcs(&acc[e], __fmaf_rn(2.0f, kf, ra));
                __stcs(&out[e], __fmaf_rn(cf.dt, kf, r0));
            } else {
                wn[f] = __fmaf_rn(cf.d6, ra + kf, r0);
                out[e] = wn[f];
            }
        }
        if (STAGE == 4) {   // signal speeds |v_d| + c_f of the new state
            const float ri = rcpf(wn[0]);
            const float vx = wn[1] * ri, vy = wn[2] * ri, vz = wn[3] * ri;
            const float b2 = __fmaf_rn(wn[7], wn[7], __fmaf_rn(wn[6], wn[6], wn[5] * wn[5]));
            const float ekin = 0.5f * __fmaf_rn(wn[3], vz, __fmaf_rn(wn[2], vy, wn[1] * vx));
            const float pk_ = (cf.gamma - 1.0f) * ((wn[4] - ekin) - 0.5f * b2);
            const float cfs = sqrtf(__fmaf_rn(cf.gamma, pk_, b2) * ri);
            const float sp[3] = {fabsf(vx) + cfs, fabsf(vy) + cfs, fabsf(vz) + cfs};
#pragma unroll
            for (int d = 0; d < 3; ++d) if (!(sp[d] <= sp_max[d])) sp_max[d] = sp[d];   // NaN propagates
        }
    }
    if (STAGE == 4) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            unsigned long long key = (unsigned long long)__double_as_longlong((double)sp_max[d]);
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long w2 = __shfl_xor_sync(0xffffffffu, key, o);
                key = w2 > key ? w2 : key;
            }
            if (lane == 0) atomicMax(&keys[d], key);
        }
    }
}

// shock indicator s = max(0, -div v) on [-1, n+1) in every direction, from the
// stage input.  One CTA owns 32 x 4 output columns and marches skz planes along
// z.  Planes of (rho, m_x, m_y, m_z) with a 2-cell x/y halo arrive by one
// tensor-map TMA copy each into a ring of SNB = 4 buffers (plane q in buffer
// q mod SNB, one mbarrier per buffer; plane k+SNB is copied once plane k is
// done); v_x and
// v_y of plane k are formed once per cell in shared memory, v_z of the own
// column at planes k .. k+2 from the ring and at k-1, k-2 from two rolled
// registers.  Same arithmetic as the per-cell form.  Every copy issued is waited
// for before the CTA leaves (bounded waits; a timeout sets *status).
struct ShSmem {
    float pl[SNB][4][SRH][SRW];   // x = 32 bx - 4 + c, y = yo - 2 + r (yo = STY by - 1)
    float vx[STY][SRW];           // v_x of the tile rows, by staged column
    float vy[SRH][STX];           // v_y of the staged rows, tile columns
};
static_assert((4 * SRH * SRW * sizeof(float)) % 128 == 0, "plane buffers 128-byte aligned");
constexpr unsigned kShPlaneBytes = (unsigned)(4 * SRH * SRW * sizeof(float));
__global__ void __launch_bounds__(SNT) shock3_f32(float* __restrict__ sh, Grid3 g, float i12x, float i12y, float i12z,
                                                  int ntx, int skz, int* __restrict__ status,
                                                  const __grid_constant__ CUtensorMap tm)
{
    __shared__ __align__(128) ShSmem S;
    __shared__ __align__(8) unsigned long long bar[SNB];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int bx = (int)(blockIdx.x % ntx), by = (int)(blockIdx.x / ntx);
    const int xo = STX * bx - 1, yo = STY * by - 1;
    const int k0 = skz * (int)blockIdx.y - 1, k1 = min(k0 + skz, g.nz + 1);
    const int x = xo + lane, y = yo + w;
    const bool valid = x <= g.nx && y <= g.ny;
    const long long P = g.ex * g.ey;
    const int c0 = lane + 3, r0 = w + 2;   // own output cell in a staged plane
    if (*status != 0) return;
    if (tid == 0)
        for (int b = 0; b < SNB; ++b) mbar_init(&bar[b]);
    __syncthreads();
    unsigned phase = 0, pending = 0;   // per buffer: parity of the next completion; copy issued, not yet waited
    const auto buf = [](int q) { return (q + SNB) % SNB; };   // q >= -3 > -SNB
    const auto issue = [&](int q) {
        const int b = buf(q);
        pending |= 1u << b;
        if (tid == 0) {
            mbar_expect_tx(&bar[b], kShPlaneBytes);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            tma4(&S.pl[b][0][0][0], &tm, STX * bx, STY * by, q + G3, 0, &bar[b]);
        }
    };
    const auto wait = [&](int q) {   // true on timeout
        const int b = buf(q);
        const bool to = !mbar_wait_bounded(&bar[b], (phase >> b) & 1u);
        phase ^= 1u << b;
        pending &= ~(1u << b);
        return to;
    };
    const auto give_up = [&]() {   // uniform: record the timeout, let copies in flight land, leave
        if (tid == 0) {
            atomicExch(status, 1);
            for (int b = 0; b < SNB; ++b)
                if (pending & (1u << b)) mbar_wait_bounded(&bar[b], (phase >> b) & 1u);
        }
    };
    const auto vz_of = [&](int b) { return S.pl[b][3][r0][c0] * rcpf(S.pl[b][0][r0][c0]); };

    // planes k0-2 .. k0+SNB-3 (never past k1+1, the last plane a step reads);
    // v_z of the first two; then k0+SNB-2, k0+SNB-1 into their buffers
    for (int q = k0 - 2; q <= k0 + SNB - 3 && q <= k1 + 1; ++q) issue(q);
    bool to = wait(k0 - 2);
    to = wait(k0 - 1) || to;
    if (__syncthreads_or(to)) { give_up(); return; }
    float vzm2 = vz_of(buf(k0 - 2)), vzm1 = vz_of(buf(k0 - 1));
    __syncthreads();   // the buffers of k0-2, k0-1 are free
    if (k0 + SNB - 2 <= k1 + 1) issue(k0 + SNB - 2);
    if (k0 + SNB - 1 <= k1 + 1) issue(k0 + SNB - 1);
#pragma unroll 1
    for (int k = k0; k < k1; ++k) {
        to = false;
        if (k == k0) { to = wait(k0); to = wait(k0 + 1) || to; }
        to = wait(k + 2) || to;
        if (__syncthreads_or(to)) { give_up(); return; }
        const int bk = buf(k);
        for (int i = tid; i < STY * (STX + 4); i += SNT) {   // v_x: tile rows, staged columns 1 .. 36
            const int r = i / (STX + 4), c = 1 + i - (i / (STX + 4)) * (STX + 4);
            S.vx[r][c] = S.pl[bk][1][r + 2][c] * rcpf(S.pl[bk][0][r + 2][c]);
        }
        for (int i = tid; i < SRH * STX; i += SNT) {          // v_y: staged rows 0 .. 7, tile columns
            const int r = i / STX, c = i - (i / STX) * STX;
            S.vy[r][c] = S.pl[bk][2][r][c + 3] * rcpf(S.pl[bk][0][r][c + 3]);
        }
        const float vz0 = vz_of(bk), vzp1 = vz_of(buf(k + 1)), vzp2 = vz_of(buf(k + 2));
        __syncthreads();
        if (valid) {
            const float* vr = &S.vx[w][c0];
            const float* vc = &S.vy[r0][lane];
            const float dvx = __fmaf_rn(8.0f, vr[1] - vr[-1], -(vr[2] - vr[-2]));
            const float dvy = __fmaf_rn(8.0f, vc[STX] - vc[-STX], -(vc[2 * STX] - vc[-2 * STX]));
            const float dvz = __fmaf_rn(8.0f, vzp1 - vzm1, -(vzp2 - vzm2));
            const float div = (dvx * i12x + dvy * i12y) + dvz * i12z;
            sh[(long long)(k + G3) * P + (long long)(y + G3) * g.ex + (x + GX)] = fmaxf(0.0f, -div);
        }
        vzm2 = vzm1; vzm1 = vz0;
        __syncthreads();   // plane k's buffer and v_x, v_y are free
        if (k + SNB <= k1 + 1) issue(k + SNB);   // into plane k's buffer
    }
}
}  // namespace f3

namespace f3 {
cudaError_t prepare()
{
    const int b = (int)sizeof(Smem);
    cudaError_t e = cudaFuncSetAttribute(stage3_f32<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(stage3_f32<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(stage3_f32<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(stage3_f32<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    return e;
}

cudaError_t launch_stage(int stage, const float* in, const float* sh, const float* u0, float* acc, float* out,
                         const Grid3& g, const Coef& cf, unsigned long long* keys, int* status, const Maps& m,
                         cudaStream_t st)
{
    const int ntx = (g.nx + TX - 1) / TX, nty = (g.ny + TY - 1) / TY;
    const dim3 grid((unsigned)(ntx * nty), (unsigned)((g.nz + cf.kz - 1) / cf.kz));
    const size_t sm = sizeof(Smem);
    switch (stage) {
        case 1: stage3_f32<1><<<grid, NT, sm, st>>>(in, sh, u0, acc, out, g, cf, ntx, keys, status, m); break;
        case 2: stage3_f32<2><<<grid, NT, sm, st>>>(in, sh, u0, acc, out, g, cf, ntx, keys, status, m); break;
        case 3: stage3_f32<3><<<grid, NT, sm, st>>>(in, sh, u0, acc, out, g, cf, ntx, keys, status, m); break;
        case 4: stage3_f32<4><<<grid, NT, sm, st>>>(in, sh, u0, acc, out, g, cf, ntx, keys, status, m); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_shock(float* sh, const Grid3& g, const Coef& cf, int sntx, dim3 grid, int* status,
                         const CUtensorMap& tm, cudaStream_t st)
{
    shock3_f32<<<grid, SNT, 0, st>>>(sh, g, cf.i12[0], cf.i12[1], cf.i12[2], sntx, cf.kz, status, tm);
    return cudaGetLastError();
}
}  // namespace f3
}  // namespace sac3d
