// sac3d.cu -- the 3D form of the split ideal-MHD RK4 step (section 2 of
// arXiv 1710.06423 written for three-component vectors): eight conserved
// fields rho, m_x, m_y, m_z, e, B_x, B_y, B_z on a periodic box, no background.
//
// FP64 (the oracle-order path; the unit is compiled without FMA contraction,
// so FP64 agrees with the FP64 3D oracle to rounding order): each RK stage
// runs four kernels in the method's own order of operations:
//   ghosts3   periodic ghost frame (3 cells; 4 on the left in x) of the stage input;
//   flux3     per ghost-extended cell: velocities and the fluxes of all eight
//             fields along x, y and z (global scratch);
//   shock3    s = max(0, -((D_x v_x + D_y v_y) + D_z v_z)) on the cells the
//             face coefficients need;
//   update3   per interior cell: k = ((H_x + H_y) + H_z) - ((D_x F_x + D_y F_y)
//             + D_z F_z) (hyper-diffusion with the maxima over three faces,
//             fourth-order flux differences) and the classical RK4 register
//             update (K = k1 + 2 k2 + 2 k3, U = U0 + dt/6 (K + k4)).
// FP32 (the performance path): ghosts3, f3::shock3_f32 and one fused stage
// kernel (f3::stage3_f32); both f3 kernels march column tiles through z fed by
// tensor-map TMA copies; stage 4 also reduces the next step's signal speeds.
// The step's signal speeds come from one reduction over the state (ordered
// bits, NaN propagates); dt = C min(min(dx/cx, dy/cy), dz/cz) is formed on
// the host in FP64.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstddef>
#include <cstring>
#include <limits>
#include <string>

#include "../../include/sac.h"

namespace {

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

__device__ __forceinline__ int wrapn(int i, int n) { int r = i % n; return r < 0 ? r + n : r; }

// periodic ghost frame: one block per extended row (y, z); ghost rows are copied
// whole from their wrapped interior row, interior rows get their x ghosts.  Only
// interior cells are read, so the copies are independent of one another.
template <typename T>
__global__ void ghosts3(T* __restrict__ s, Grid3 g)
{
    const int row = blockIdx.x;                       // 0 .. ey*ez - 1
    const int j = row % (int)g.ey - G3, k = row / (int)g.ey - G3;
    const bool ghost_row = j < 0 || j >= g.ny || k < 0 || k >= g.nz;
    const long long dst = (long long)row * g.ex;
    const long long src = ((long long)(wrapn(k, g.nz) + G3) * g.ey + (wrapn(j, g.ny) + G3)) * g.ex;
    const int nxg = (int)g.ex - g.nx;                 // GX on the left, the rest on the right
    const int cnt = ghost_row ? (int)g.ex : nxg;
    for (int t = threadIdx.x; t < cnt * NF3; t += blockDim.x) {
        const int f = t / cnt, q = t - f * cnt;
        const int xi = ghost_row ? q : (q < GX ? q : g.nx + q);
        T* u = s + (long long)f * g.ne;
        u[dst + xi] = u[src + wrapn(xi - GX, g.nx) + GX];
    }
}

// velocities v[3][ne] and fluxes fl[3][8][ne] at every ghost-extended cell
template <typename T>
__global__ void flux3(const T* __restrict__ s, T* __restrict__ v, T* __restrict__ fl, Grid3 g, T gm1)
{
    const long long ne = g.ne;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ne; c += (long long)gridDim.x * blockDim.x) {
        const T rho = s[c], mx = s[ne + c], my = s[2 * ne + c], mz = s[3 * ne + c], et = s[4 * ne + c];
        const T bx = s[5 * ne + c], by = s[6 * ne + c], bz = s[7 * ne + c];
        const T ux = mx / rho, uy = my / rho, uz = mz / rho;
        const T ekin = (T)0.5 * ((mx * ux + my * uy) + mz * uz);
        const T b2 = (T)0.5 * ((bx * bx + by * by) + bz * bz);
        const T pk = gm1 * ((et - ekin) - b2);
        const T pt = pk + b2;
        const T bv = (bx * ux + by * uy) + bz * uz;
        const T etot = et + pt;
        v[c] = ux; v[ne + c] = uy; v[2 * ne + c] = uz;
        const T ud[3] = {ux, uy, uz}, bd[3] = {bx, by, bz}, md[3] = {mx, my, mz};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            T* F = fl + (long long)d * NF3 * ne;
            F[c] = md[d];
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                const T f = ud[d] * md[q] - bd[d] * bd[q];
                F[(1 + q) * ne + c] = (q == d) ? f + pt : f;
            }
            F[4 * ne + c] = ud[d] * etot - bd[d] * bv;
#pragma unroll
            for (int q = 0; q < 3; ++q) F[(5 + q) * ne + c] = ud[d] * bd[q] - bd[d] * ud[q];
        }
    }
}

template <typename T>
__device__ __forceinline__ T dcen3(const T* f, long long c, long long s, T d12)
{
    return ((T)8.0 * (f[c + s] - f[c - s]) - (f[c + 2 * s] - f[c - 2 * s])) / d12;
}

// shock indicator on [-1, n+1) in every direction
template <typename T>
__global__ void shock3(const T* __restrict__ v, T* __restrict__ sh, Grid3 g, T d12x, T d12y, T d12z)
{
    const long long bx = g.nx + 2, by = g.ny + 2, bz = g.nz + 2, tot = bx * by * bz;
    const long long sy = g.ex, sz = g.ex * g.ey;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(t % bx) - 1, j = (int)((t / bx) % by) - 1, k = (int)(t / (bx * by)) - 1;
        const long long c = g.at(i, j, k);
        const T div = (dcen3(v, c, 1, d12x) + dcen3(v + g.ne, c, sy, d12y)) + dcen3(v + 2 * g.ne, c, sz, d12z);
        sh[c] = fmax((T)0, -div);
    }
}

struct Coef3 {
    double c2[NF3];
    double c_shk;
    double dd[3];
    double cm[3];
    int hd;
};

// k of every field at every interior cell, then the RK register update
template <typename T, int STAGE>
__global__ void update3(const T* __restrict__ s, const T* __restrict__ fl, const T* __restrict__ sh,
                        T* u0, T* __restrict__ acc, T* out, Grid3 g, Coef3 cf,   // out == u0 in stage 4
                        T dt, T h, T d6)
{
    const long long n = (long long)g.nx * g.ny * g.nz;
    const long long st[3] = {1, g.ex, g.ex * g.ey};
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(t % g.nx), j = (int)((t / g.nx) % g.ny), k = (int)(t / ((long long)g.nx * g.ny));
        const long long c = g.at(i, j, k);
#pragma unroll 1
        for (int f = 0; f < NF3; ++f) {
            const T* uf = s + (long long)f * g.ne;
            T hsum = (T)0;
            if (cf.hd) {
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    const long long S = st[d];
                    const T a = (T)((cf.c2[f] * cf.dd[d]) * cf.cm[d]);
                    const T bsh = (T)((cf.c_shk * cf.dd[d]) * cf.dd[d]);
                    T gf[2];
#pragma unroll
                    for (int side = 0; side < 2; ++side) {
                        const long long fc = side ? c : c - S;
                        T a1[3], a3[3], d1c = (T)0;
#pragma unroll
                        for (int o = -1; o <= 1; ++o) {
                            const long long q = fc + o * S;
                            const T d1 = uf[q + S] - uf[q];
                            const T d3 = (uf[q + 2 * S] - uf[q - S]) - (T)3.0 * d1;
                            a1[o + 1] = fabs(d1); a3[o + 1] = fabs(d3);
                            if (o == 0) d1c = d1;
                        }
                        const T m1 = fmax(fmax(a1[0], a1[1]), a1[2]);
                        const T m3 = fmax(fmax(a3[0], a3[1]), a3[2]);
                        const T r = (m1 > (T)0) ? m3 / m1 : (T)0;
                        const T sf = (T)0.5 * (sh[fc] + sh[fc + S]);
                        const T nu = a * r + bsh * sf;
                        gf[side] = nu * d1c;
                    }
                    const T dd = (T)cf.dd[d];
                    hsum = hsum + (gf[1] - gf[0]) / (dd * dd);
                }
            }
            const T dfx = dcen3(fl + (0 * NF3 + f) * g.ne, c, st[0], (T)(12.0 * cf.dd[0]));
            const T dfy = dcen3(fl + (1 * NF3 + f) * g.ne, c, st[1], (T)(12.0 * cf.dd[1]));
            const T dfz = dcen3(fl + (2 * NF3 + f) * g.ne, c, st[2], (T)(12.0 * cf.dd[2]));
            const T kf = hsum - ((dfx + dfy) + dfz);
            const long long e = (long long)f * g.ne + c;
            if (STAGE == 1) {
                acc[e] = kf;
                out[e] = u0[e] + h * kf;
            } else if (STAGE == 2) {
                acc[e] = acc[e] + (T)2.0 * kf;
                out[e] = u0[e] + h * kf;
            } else if (STAGE == 3) {
                acc[e] = acc[e] + (T)2.0 * kf;
                out[e] = u0[e] + dt * kf;
            } else {
                out[e] = u0[e] + d6 * (acc[e] + kf);   // out is U0 itself: pointwise
            }
        }
    }
}

// signal speeds |v_d| + c_f, maximum over the interior; blocks stride over the
// (y, z) rows, threads over x; one ordered-bit atomic per warp and direction
template <typename T>
__global__ void cmax3_kernel(const T* __restrict__ s, Grid3 g, T gamma, unsigned long long* __restrict__ keys)
{
    const long long ne = g.ne;
    const int rows = g.ny * g.nz;
    double mxs[3] = {0.0, 0.0, 0.0};
    for (int r = blockIdx.x; r < rows; r += gridDim.x) {
        const int j = r % g.ny, k = r / g.ny;
        for (int i = threadIdx.x; i < g.nx; i += blockDim.x) {
            const long long c = g.at(i, j, k);
            const T rho = s[c], mx = s[ne + c], my = s[2 * ne + c], mz = s[3 * ne + c], et = s[4 * ne + c];
            const T bx = s[5 * ne + c], by = s[6 * ne + c], bz = s[7 * ne + c];
            const T ux = mx / rho, uy = my / rho, uz = mz / rho;
            const T ekin = (T)0.5 * ((mx * ux + my * uy) + mz * uz);
            const T b2 = (T)0.5 * ((bx * bx + by * by) + bz * bz);
            const T pk = (gamma - (T)1) * ((et - ekin) - b2);
            const T cfst = sqrt((gamma * pk + ((bx * bx + by * by) + bz * bz)) / rho);
            const double sp[3] = {(double)(fabs(ux) + cfst), (double)(fabs(uy) + cfst), (double)(fabs(uz) + cfst)};
#pragma unroll
            for (int d = 0; d < 3; ++d) if (!(sp[d] <= mxs[d])) mxs[d] = sp[d];   // NaN propagates
        }
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        unsigned long long key = (unsigned long long)__double_as_longlong(mxs[d]);
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long w = __shfl_xor_sync(0xffffffffu, key, o);
            key = w > key ? w : key;
        }
        if ((threadIdx.x & 31) == 0) atomicMax(&keys[d], key);
    }
}

// FP64 diagnostics of the current state, in a fixed reduction order: the
// eight field sums over the interior, and the discrete div B = Dx Bx + Dy By +
// Dz Bz with section 2's fourth-order central difference (neighbours wrapped
// across the periodic box), as sum |div B| and max |div B|.  Per block:
// part[b][0..7] field sums, [8] sum |div B|, [9] max |div B|.
constexpr int kDiagBlocks = 296, kDiagVals = NF3 + 2;
// maximum that keeps a NaN (fmax would drop it)
__device__ inline double max_nan3(double a, double b) { return (a > b || a != a) ? a : b; }
template <typename T>
__global__ void __launch_bounds__(256) diag3_partial(const T* __restrict__ s, Grid3 g, double i12x, double i12y,
                                                     double i12z, double* __restrict__ part)
{
    __shared__ double red[kDiagVals][8];
    double acc[NF3 + 1], mx = 0.0;
#pragma unroll
    for (int f = 0; f <= NF3; ++f) acc[f] = 0.0;
    const long long n = (long long)g.nx * g.ny * g.nz;
    const auto b = [&](int f, int i, int j, int k) { return (double)s[(long long)f * g.ne + g.at(i, j, k)]; };
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(v % g.nx);
        const long long r = v / g.nx;
        const int j = (int)(r % g.ny), k = (int)(r / g.ny);
#pragma unroll
        for (int f = 0; f < NF3; ++f) acc[f] += b(f, i, j, k);
        const int xm2 = wrapn(i - 2, g.nx), xm1 = wrapn(i - 1, g.nx), xp1 = wrapn(i + 1, g.nx), xp2 = wrapn(i + 2, g.nx);
        const int ym2 = wrapn(j - 2, g.ny), ym1 = wrapn(j - 1, g.ny), yp1 = wrapn(j + 1, g.ny), yp2 = wrapn(j + 2, g.ny);
        const int zm2 = wrapn(k - 2, g.nz), zm1 = wrapn(k - 1, g.nz), zp1 = wrapn(k + 1, g.nz), zp2 = wrapn(k + 2, g.nz);
        const double dxb = (b(5, xm2, j, k) - 8.0 * b(5, xm1, j, k) + 8.0 * b(5, xp1, j, k) - b(5, xp2, j, k)) * i12x;
        const double dyb = (b(6, i, ym2, k) - 8.0 * b(6, i, ym1, k) + 8.0 * b(6, i, yp1, k) - b(6, i, yp2, k)) * i12y;
        const double dzb = (b(7, i, j, zm2) - 8.0 * b(7, i, j, zm1) + 8.0 * b(7, i, j, zp1) - b(7, i, j, zp2)) * i12z;
        const double a = fabs((dxb + dyb) + dzb);
        acc[NF3] += a;
        mx = max_nan3(mx, a);
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < kDiagVals; ++q) {
        double x = q <= NF3 ? acc[q] : mx;
        for (int o = 16; o > 0; o >>= 1) {
            const double y = __shfl_xor_sync(0xffffffffu, x, o);
            x = q <= NF3 ? x + y : max_nan3(x, y);
        }
        if (lane == 0) red[q][w] = x;
    }
    __syncthreads();
    if (threadIdx.x < kDiagVals) {
        const int q = threadIdx.x;
        double x = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) x = q <= NF3 ? x + red[q][k] : max_nan3(x, red[q][k]);
        part[blockIdx.x * kDiagVals + q] = x;
    }
}
__global__ void diag3_final(const double* __restrict__ part, int nb, double* __restrict__ out)
{
    const int q = threadIdx.x;
    if (q < kDiagVals) {
        double x = 0.0;
        for (int k = 0; k < nb; ++k) x = q <= NF3 ? x + part[k * kDiagVals + q] : max_nan3(x, part[k * kDiagVals + q]);
        out[q] = x;
    }
}

// FP64 host copy [8][nz][ny][nx] <-> extended device field (interior), converting to T
template <typename T>
__global__ void import3(const double* __restrict__ w, T* __restrict__ u, Grid3 g)
{
    const long long n = (long long)g.nx * g.ny * g.nz;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n * NF3; t += (long long)gridDim.x * blockDim.x) {
        const int f = (int)(t / n);
        const long long r = t - f * n;
        const int i = (int)(r % g.nx), j = (int)((r / g.nx) % g.ny), k = (int)(r / ((long long)g.nx * g.ny));
        u[(long long)f * g.ne + g.at(i, j, k)] = (T)w[t];
    }
}
template <typename T>
__global__ void export3(const T* __restrict__ u, double* __restrict__ w, Grid3 g)
{
    const long long n = (long long)g.nx * g.ny * g.nz;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n * NF3; t += (long long)gridDim.x * blockDim.x) {
        const int f = (int)(t / n);
        const long long r = t - f * n;
        const int i = (int)(r % g.nx), j = (int)((r / g.nx) % g.ny), k = (int)(r / ((long long)g.nx * g.ny));
        w[t] = (double)u[(long long)f * g.ne + g.at(i, j, k)];
    }
}

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
constexpr int TX = 32, TY = 4, NT = TX * TY;   // one warp per y row of the tile
constexpr int HXS = 4, RW = TX + 2 * HXS;      // staged x range i0-4 .. i0+TX+3
constexpr int RH = TY + 2 * G3;                // staged rows j0-3 .. j0+TY+2
constexpr int NS = NF3 + 1;                    // eight fields and the shock indicator
constexpr int FXW = TX + 4, FYH = TY + 4;      // flux extents: x i0-2 .. i0+TX+1, y j0-2 .. j0+TY+1

struct Smem {
    float full[2][NS + 1][RH][RW];   // planes k and k+1 (one spare field-plane: 128-byte aligned buffers)
    float col[4][NS][NT];        // planes k+1 .. k+4, own column (ring by plane % 4)
    float fz[5][NF3][NT];     // z fluxes of planes k-2 .. k+2, own column (ring by plane % 5)
    float fx[NF3][TY][FXW];
    float fy[NF3][FYH][TX];
    float rk[2][2][NF3][NT];     // U0 and the RK accumulator of the own cell, planes k and k+1
    float hy[NF3][TY][TX];       // y hyper-diffusion of plane k (the y sweep of phase 1)
};

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

__device__ __forceinline__ float rcpf(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
// tensor maps of one stage launch: the stage input (4D: x, y, z, field) and the
// shock indicator (3D) as a staged plane box and as a column-tile box, U0 and
// the RK accumulator as column-tile boxes
struct Maps {
    CUtensorMap in_full, in_col, sh_full, sh_col, u0_col, acc_col;
};
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
// tensor-map TMA copy each into a ring of four buffers (plane q in buffer q mod
// 4, one mbarrier per buffer; plane k+4 is copied once plane k is done); v_x and
// v_y of plane k are formed once per cell in shared memory, v_z of the own
// column at planes k .. k+2 from the ring and at k-1, k-2 from two rolled
// registers.  Same arithmetic as the per-cell form.  Every copy issued is waited
// for before the CTA leaves (bounded waits; a timeout sets *status).
constexpr int STX = 32, STY = 4, SNT = STX * STY, SRW = 40, SRH = STY + 4, SNB = 4;
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
    const auto buf = [](int q) { return (q + SNB) % SNB; };   // q >= -3
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

    // planes k0-2 .. k0+1; v_z of the first two; then k0+2, k0+3 into their buffers
    for (int q = k0 - 2; q <= k0 + 1; ++q) issue(q);
    bool to = wait(k0 - 2);
    to = wait(k0 - 1) || to;
    if (__syncthreads_or(to)) { give_up(); return; }
    float vzm2 = vz_of(buf(k0 - 2)), vzm1 = vz_of(buf(k0 - 1));
    __syncthreads();   // the buffers of k0-2, k0-1 are free
    issue(k0 + 2);     // read at step k0 (k1 >= k0 + 1)
    if (k0 + 3 <= k1 + 1) issue(k0 + 3);
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
        if (k + 4 <= k1 + 1) issue(k + 4);   // read at step k+2 as its plane +2
    }
}
}  // namespace f3

int grid_for(long long n) { long long b = (n + 255) / 256; return (int)(b < 4096 ? (b < 1 ? 1 : b) : 4096); }

}  // namespace

struct sac3_ctx {
    sac3_params p;
    Grid3 g;
    int fp32 = 0;
    size_t esz = 8;
    cudaStream_t stream = nullptr;
    void *u0 = nullptr, *sa = nullptr, *sb = nullptr, *acc = nullptr, *v = nullptr, *fl = nullptr, *sh = nullptr;
    double* wbuf = nullptr;                 // device FP64 staging of a host state
    unsigned long long* keys = nullptr;     // signal-speed keys (3)
    int* status = nullptr;                  // FP32 stage kernels: 1 = a copy wait timed out
    double* diag = nullptr;                 // diagnostics: per-block partials, then the totals
    CUtensorMap m_full[3], m_col[3];        // FP32: stage inputs U0, SA, SB (plane box, column box)
    CUtensorMap m_sh_full, m_sh_col, m_acc_col;
    CUtensorMap m_shk[3];                   // FP32 stage inputs as (rho, m) planes of the shock kernel
    double t = 0.0;
    bool have_state = false;
    bool keys_valid = false;                // keys hold the maxima of the current state
    int drop_copies = 0;                    // test hook of the bounded copy waits
    std::string err;
};

static int fail3(sac3_ctx* c, int code, const char* fmt, ...)
{
    if (c) {
        char buf[256];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        c->err = buf;
    }
    return code;
}

#define CK3(call)                                                                         \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) return fail3(c, SAC_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

// FP32: ghost frame, shock indicator and one fused kernel per stage
template <int S>
static cudaError_t launch_f32(const float* in, const float* sh, const float* u0, float* acc, float* out,
                              const Grid3& g, const f3::Coef& cf, unsigned long long* keys, int* status,
                              const f3::Maps& m, cudaStream_t st)
{
    const int ntx = (g.nx + f3::TX - 1) / f3::TX, nty = (g.ny + f3::TY - 1) / f3::TY;
    const dim3 grid((unsigned)(ntx * nty), (unsigned)((g.nz + cf.kz - 1) / cf.kz));
    f3::stage3_f32<S><<<grid, f3::NT, sizeof(f3::Smem), st>>>(in, sh, u0, acc, out, g, cf, ntx, keys, status, m);
    return cudaGetLastError();
}

// Tensor maps of the FP32 registers: 4D (x, y, z, field) for the eight-field
// arrays, 3D for the shock indicator; box = a staged plane (40 x 10 x 1) or a
// column tile (32 x 4 x 1), all fields at once.
static bool encode_maps3(sac3_ctx* c)
{
    // looked up once (thread-safe initialisation of a function-local static)
    static const PFN_cuTensorMapEncodeTiled_v12000 encode = [] {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            fn = nullptr;
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }();
    if (!encode) return false;
    const Grid3& g = c->g;
    const cuuint64_t dims[4] = {(cuuint64_t)g.ex, (cuuint64_t)g.ey, (cuuint64_t)g.ez, (cuuint64_t)NF3};
    const cuuint64_t str[3] = {(cuuint64_t)g.ex * 4, (cuuint64_t)(g.ex * g.ey) * 4, (cuuint64_t)g.ne * 4};
    const cuuint32_t bfull[4] = {(cuuint32_t)f3::RW, (cuuint32_t)f3::RH, 1, (cuuint32_t)NF3};
    const cuuint32_t bcol[4] = {(cuuint32_t)f3::TX, (cuuint32_t)f3::TY, 1, (cuuint32_t)NF3};
    const cuuint32_t es[4] = {1, 1, 1, 1};
    const auto enc = [&](CUtensorMap* m, void* base, int rank, const cuuint32_t* box) {
        return encode(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, rank, base, dims, str, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                      CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    };
    void* regs[3] = {c->u0, c->sa, c->sb};
    bool ok = true;
    for (int r = 0; r < 3 && ok; ++r) ok = enc(&c->m_full[r], regs[r], 4, bfull) && enc(&c->m_col[r], regs[r], 4, bcol);
    ok = ok && enc(&c->m_sh_full, c->sh, 3, bfull) && enc(&c->m_sh_col, c->sh, 3, bcol) && enc(&c->m_acc_col, c->acc, 4, bcol);
    const cuuint32_t bshk[4] = {(cuuint32_t)f3::SRW, (cuuint32_t)f3::SRH, 1, 4};
    for (int r = 0; r < 3 && ok; ++r) ok = enc(&c->m_shk[r], regs[r], 4, bshk);
    return ok;
}

static cudaError_t prepare_f32()
{
    const int b = (int)sizeof(f3::Smem);
    cudaError_t e = cudaFuncSetAttribute(f3::stage3_f32<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(f3::stage3_f32<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(f3::stage3_f32<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(f3::stage3_f32<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    return e;
}

static int fused_f32(sac3_ctx* c, double dt, const double cm[3], const double dd[3], double* dt_taken)
{
    const Grid3& g = c->g;
    f3::Coef cf;
    for (int f = 0; f < NF3; ++f)
        for (int d = 0; d < 3; ++d) cf.a[f][d] = (float)(c->p.c2[f] * dd[d] * cm[d]);
    for (int d = 0; d < 3; ++d) {
        cf.bsh[d] = (float)(0.5 * c->p.c_shk * dd[d] * dd[d]);
        cf.i12[d] = (float)(1.0 / (12.0 * dd[d]));
        cf.idd[d] = (float)(1.0 / (dd[d] * dd[d]));
    }
    cf.gm1 = (float)(c->p.gamma - 1.0);
    cf.gamma = (float)c->p.gamma;
    cf.dt = (float)dt; cf.h = (float)(0.5 * dt); cf.d6 = (float)(dt / 6.0);
    cf.hd = c->p.hyperdiffusion != 0;
    cf.drop = c->drop_copies;
    {   // z chunk: 64 planes when that still leaves at least four CTAs per resident slot
        // (2 per SM), else 32 (longer chunks repeat the 6-plane prologue less often)
        const long long cols = (long long)((g.nx + f3::TX - 1) / f3::TX) * ((g.ny + f3::TY - 1) / f3::TY);
        int nsm = 148, dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        cf.kz = cols * ((g.nz + 63) / 64) >= 4LL * 2 * nsm ? 64 : 32;
    }
    float* u0 = (float*)c->u0;
    float* sa = (float*)c->sa;
    float* sb = (float*)c->sb;
    float* sh = (float*)c->sh;
    float* acc = (float*)c->acc;
    const int sntx = (g.nx + 2 + f3::STX - 1) / f3::STX, snty = (g.ny + 2 + f3::STY - 1) / f3::STY;
    const dim3 sgrid((unsigned)(sntx * snty), (unsigned)((g.nz + 2 + cf.kz - 1) / cf.kz));
    for (int stage = 1; stage <= 4; ++stage) {
        float* in = stage == 1 ? u0 : (stage == 2 ? sa : (stage == 3 ? sb : sa));
        float* out = stage == 1 ? sa : (stage == 2 ? sb : (stage == 3 ? sa : u0));
        ghosts3<float><<<(int)(g.ey * g.ez), 128, 0, c->stream>>>(in, g);
        const int ri = stage == 1 ? 0 : (stage == 3 ? 2 : 1);   // input register: U0, SA, SB, SA
        if (cf.hd)
            f3::shock3_f32<<<sgrid, f3::SNT, 0, c->stream>>>(sh, g, cf.i12[0], cf.i12[1], cf.i12[2], sntx, cf.kz, c->status,
                                                           c->m_shk[ri]);
        // stage 4 reduces the signal speeds of the new state for the next step
        if (stage == 4) CK3(cudaMemsetAsync(c->keys, 0, 3 * sizeof(unsigned long long), c->stream));
        const f3::Maps m{c->m_full[ri], c->m_col[ri], c->m_sh_full, c->m_sh_col, c->m_col[0], c->m_acc_col};
        cudaError_t e;
        switch (stage) {
            case 1: e = launch_f32<1>(in, sh, u0, acc, out, g, cf, c->keys, c->status, m, c->stream); break;
            case 2: e = launch_f32<2>(in, sh, u0, acc, out, g, cf, c->keys, c->status, m, c->stream); break;
            case 3: e = launch_f32<3>(in, sh, u0, acc, out, g, cf, c->keys, c->status, m, c->stream); break;
            default: e = launch_f32<4>(in, sh, u0, acc, out, g, cf, c->keys, c->status, m, c->stream); break;
        }
        CK3(e);
    }
    int st = 0;
    CK3(cudaMemcpyAsync(&st, c->status, sizeof st, cudaMemcpyDeviceToHost, c->stream));
    CK3(cudaStreamSynchronize(c->stream));
    if (st != 0) {
        // the step is abandoned (U0 is written only by a completed stage 4); the next step retries
        CK3(cudaMemsetAsync(c->status, 0, sizeof(int), c->stream));
        CK3(cudaStreamSynchronize(c->stream));
        c->keys_valid = false;
        return fail3(c, SAC_ERR_TIMEOUT, "a stage kernel's copy wait timed out");
    }
    c->keys_valid = true;
    c->t += dt;
    if (dt_taken) *dt_taken = dt;
    return SAC_OK;
}

template <typename T>
static int step3(sac3_ctx* c, double dt_in, double* dt_taken)
{
    const Grid3& g = c->g;
    const long long n = (long long)g.nx * g.ny * g.nz;
    const double dd[3] = {(c->p.x1 - c->p.x0) / g.nx, (c->p.y1 - c->p.y0) / g.ny, (c->p.z1 - c->p.z0) / g.nz};
    // signal speeds of the step-start state (all four stages use them)
    // (the FP32 stage 4 leaves the maxima of its output in keys)
    if (!c->keys_valid) {
        CK3(cudaMemsetAsync(c->keys, 0, 3 * sizeof(unsigned long long), c->stream));
        const int crow = g.ny * g.nz < 148 * 8 ? g.ny * g.nz : 148 * 8;
        cmax3_kernel<T><<<crow, 128, 0, c->stream>>>((const T*)c->u0, g, (T)c->p.gamma, c->keys);
        CK3(cudaGetLastError());
    }
    c->keys_valid = false;
    unsigned long long hk[3];
    CK3(cudaMemcpyAsync(hk, c->keys, sizeof hk, cudaMemcpyDeviceToHost, c->stream));
    CK3(cudaStreamSynchronize(c->stream));
    double cm[3];
    for (int d = 0; d < 3; ++d) { long long b; memcpy(&b, &hk[d], 8); double x; memcpy(&x, &b, 8); cm[d] = x; }
    double dt = dt_in > 0.0 ? dt_in : c->p.courant * fmin(fmin(dd[0] / cm[0], dd[1] / cm[1]), dd[2] / cm[2]);
    if (!(dt > 0.0) || !std::isfinite(dt) || !std::isfinite(cm[0]) || !std::isfinite(cm[1]) || !std::isfinite(cm[2]))
        return fail3(c, SAC_ERR_NONFINITE, "non-finite state or step at t = %g", c->t);
    if (c->fp32) return fused_f32(c, dt, cm, dd, dt_taken);
    Coef3 cf;
    for (int f = 0; f < NF3; ++f) cf.c2[f] = c->p.c2[f];
    cf.c_shk = c->p.c_shk;
    for (int d = 0; d < 3; ++d) { cf.dd[d] = dd[d]; cf.cm[d] = cm[d]; }
    cf.hd = c->p.hyperdiffusion != 0;
    const T gm1 = (T)(c->p.gamma - 1.0);
    const T Tdt = (T)dt, Th = (T)(0.5 * dt), Td6 = (T)(dt / 6.0);
    // stage inputs / outputs: U0 -> SA -> SB -> SA -> (U0 updated pointwise)
    T* u0 = (T*)c->u0;
    T* sa = (T*)c->sa;
    T* sb = (T*)c->sb;
    for (int stage = 1; stage <= 4; ++stage) {
        T* in = stage == 1 ? u0 : (stage == 2 ? sa : (stage == 3 ? sb : sa));
        T* out = stage == 1 ? sa : (stage == 2 ? sb : (stage == 3 ? sa : u0));
        ghosts3<T><<<(int)(g.ey * g.ez), 128, 0, c->stream>>>(in, g);
        flux3<T><<<grid_for(g.ne), 256, 0, c->stream>>>(in, (T*)c->v, (T*)c->fl, g, gm1);
        if (cf.hd)
            shock3<T><<<grid_for((long long)(g.nx + 2) * (g.ny + 2) * (g.nz + 2)), 256, 0, c->stream>>>(
                (const T*)c->v, (T*)c->sh, g, (T)(12.0 * dd[0]), (T)(12.0 * dd[1]), (T)(12.0 * dd[2]));
        const T* fl = (const T*)c->fl;
        const T* sh = (const T*)c->sh;
        T* acc = (T*)c->acc;
        switch (stage) {
            case 1: update3<T, 1><<<grid_for(n), 256, 0, c->stream>>>(in, fl, sh, u0, acc, out, g, cf, Tdt, Th, Td6); break;
            case 2: update3<T, 2><<<grid_for(n), 256, 0, c->stream>>>(in, fl, sh, u0, acc, out, g, cf, Tdt, Th, Td6); break;
            case 3: update3<T, 3><<<grid_for(n), 256, 0, c->stream>>>(in, fl, sh, u0, acc, out, g, cf, Tdt, Th, Td6); break;
            default: update3<T, 4><<<grid_for(n), 256, 0, c->stream>>>(in, fl, sh, u0, acc, out, g, cf, Tdt, Th, Td6); break;
        }
        CK3(cudaGetLastError());
    }
    CK3(cudaStreamSynchronize(c->stream));
    c->t += dt;
    if (dt_taken) *dt_taken = dt;
    return SAC_OK;
}

extern "C" {

void sac3_default_params(sac3_params* p)
{
    if (!p) return;
    memset(p, 0, sizeof(*p));
    p->nx = p->ny = p->nz = 32;
    p->x1 = p->y1 = p->z1 = 1.0;
    p->gamma = 5.0 / 3.0; p->courant = 0.3;
    p->precision = SAC_FP64;
    p->hyperdiffusion = 1;
    const double c2[8] = {0.02, 0.1, 0.1, 0.1, 0.02, 0.02, 0.02, 0.02};
    for (int f = 0; f < 8; ++f) p->c2[f] = c2[f];
    p->c_shk = 0.5;
}

const char* sac3_last_error(const sac3_ctx* c) { return c ? c->err.c_str() : "null context"; }

void sac3_free(sac3_ctx* c)
{
    if (!c) return;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(c->p.device);
    cudaFree(c->u0); cudaFree(c->sa); cudaFree(c->sb); cudaFree(c->acc); cudaFree(c->v); cudaFree(c->fl); cudaFree(c->sh);
    cudaFree(c->wbuf); cudaFree(c->keys); cudaFree(c->status); cudaFree(c->diag);
    cudaSetDevice(prev);
    delete c;
}

int sac3_init(const sac3_params* p, sac3_ctx** out)
{
    if (out) *out = nullptr;
    if (!p || !out) return SAC_ERR_ARG;
    if (p->nx < 1 || p->ny < 1 || p->nz < 1 || p->nx > 4096 || p->ny > 4096 || p->nz > 4096) return SAC_ERR_ARG;
    if (!(p->x1 > p->x0) || !(p->y1 > p->y0) || !(p->z1 > p->z0) || !(p->gamma > 1.0) || !(p->courant > 0.0))
        return SAC_ERR_ARG;
    if (p->precision != SAC_FP64 && p->precision != SAC_FP32) return SAC_ERR_ARG;
    for (int f = 0; f < 8; ++f) if (!(p->c2[f] >= 0.0)) return SAC_ERR_ARG;
    if (!(p->c_shk >= 0.0)) return SAC_ERR_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || p->device < 0 || p->device >= ndev) return SAC_ERR_ARG;
    sac3_ctx* c = new sac3_ctx();
    c->p = *p;
    c->fp32 = p->precision == SAC_FP32;
    c->esz = c->fp32 ? 4 : 8;
    c->stream = (cudaStream_t)p->stream;
    Grid3& g = c->g;
    g.nx = p->nx; g.ny = p->ny; g.nz = p->nz;
    g.ex = (p->nx + 2 * GX + 3) / 4 * 4; g.ey = p->ny + 2 * G3; g.ez = p->nz + 2 * G3;
    g.ne = g.ex * g.ey * g.ez;
    const long long n = (long long)p->nx * p->ny * p->nz;
    int rc = SAC_OK;
    if (cudaSetDevice(p->device) != cudaSuccess) rc = fail3(c, SAC_ERR_CUDA, "cudaSetDevice");
    const size_t fb = (size_t)g.ne * c->esz;
    if (rc == SAC_OK &&
        (cudaMalloc(&c->u0, NF3 * fb) != cudaSuccess || cudaMalloc(&c->sa, NF3 * fb) != cudaSuccess ||
         cudaMalloc(&c->sb, NF3 * fb) != cudaSuccess ||
         cudaMalloc(&c->acc, NF3 * fb) != cudaSuccess || cudaMalloc(&c->sh, fb) != cudaSuccess ||
         // velocity and flux scratch of the FP64 kernels
         (!c->fp32 && (cudaMalloc(&c->v, 3 * fb) != cudaSuccess || cudaMalloc(&c->fl, 3 * NF3 * fb) != cudaSuccess)) ||
         cudaMalloc(&c->wbuf, (size_t)NF3 * n * sizeof(double)) != cudaSuccess ||
         cudaMalloc(&c->keys, 3 * sizeof(unsigned long long)) != cudaSuccess ||
         cudaMalloc(&c->status, sizeof(int)) != cudaSuccess ||
         cudaMalloc(&c->diag, (size_t)(kDiagBlocks + 1) * kDiagVals * sizeof(double)) != cudaSuccess)) {
        cudaGetLastError();
        rc = fail3(c, SAC_ERR_OOM, "device allocation failed");
    }
    if (rc == SAC_OK && (cudaMemset(c->u0, 0, NF3 * fb) != cudaSuccess || cudaMemset(c->sa, 0, NF3 * fb) != cudaSuccess ||
                         cudaMemset(c->sb, 0, NF3 * fb) != cudaSuccess || cudaMemset(c->sh, 0, fb) != cudaSuccess))
        rc = fail3(c, SAC_ERR_CUDA, "cudaMemset");
    if (rc == SAC_OK && c->fp32 && prepare_f32() != cudaSuccess) rc = fail3(c, SAC_ERR_CUDA, "cudaFuncSetAttribute");
    if (rc == SAC_OK && cudaMemset(c->status, 0, sizeof(int)) != cudaSuccess) rc = fail3(c, SAC_ERR_CUDA, "cudaMemset");
    if (rc == SAC_OK && c->fp32 && !encode_maps3(c)) rc = fail3(c, SAC_ERR_CUDA, "tensor maps of the FP32 registers");
    if (rc != SAC_OK) { sac3_free(c); return rc; }
    *out = c;
    return SAC_OK;
}

int sac3_set_state(sac3_ctx* c, const double* w, double t)
{
    if (!c || !w || !std::isfinite(t)) return fail3(c, SAC_ERR_ARG, "bad arguments");
    CK3(cudaSetDevice(c->p.device));
    const long long n = (long long)c->g.nx * c->g.ny * c->g.nz;
    CK3(cudaMemcpyAsync(c->wbuf, w, (size_t)NF3 * n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    if (c->fp32) import3<float><<<grid_for(n * NF3), 256, 0, c->stream>>>(c->wbuf, (float*)c->u0, c->g);
    else import3<double><<<grid_for(n * NF3), 256, 0, c->stream>>>(c->wbuf, (double*)c->u0, c->g);
    CK3(cudaGetLastError());
    CK3(cudaStreamSynchronize(c->stream));
    c->t = t;
    c->have_state = true;
    c->keys_valid = false;
    return SAC_OK;
}

int sac3_get_state(sac3_ctx* c, double* w, double* t)
{
    if (!c || !w) return fail3(c, SAC_ERR_ARG, "bad arguments");
    if (!c->have_state) return fail3(c, SAC_ERR_STATE, "no state set");
    CK3(cudaSetDevice(c->p.device));
    const long long n = (long long)c->g.nx * c->g.ny * c->g.nz;
    if (c->fp32) export3<float><<<grid_for(n * NF3), 256, 0, c->stream>>>((const float*)c->u0, c->wbuf, c->g);
    else export3<double><<<grid_for(n * NF3), 256, 0, c->stream>>>((const double*)c->u0, c->wbuf, c->g);
    CK3(cudaGetLastError());
    CK3(cudaMemcpyAsync(w, c->wbuf, (size_t)NF3 * n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK3(cudaStreamSynchronize(c->stream));
    if (t) *t = c->t;
    return SAC_OK;
}

int sac3_step(sac3_ctx* c, double dt, double* dt_taken)
{
    if (!c) return SAC_ERR_ARG;
    if (!c->have_state) return fail3(c, SAC_ERR_STATE, "no state set");
    if (!(dt <= 0.0) && !std::isfinite(dt)) return fail3(c, SAC_ERR_ARG, "dt must be finite");
    CK3(cudaSetDevice(c->p.device));
    return c->fp32 ? step3<float>(c, dt, dt_taken) : step3<double>(c, dt, dt_taken);
}

int sac3_steps(sac3_ctx* c, long n)
{
    if (!c || n < 0) return SAC_ERR_ARG;
    for (long k = 0; k < n; ++k) {
        const int rc = sac3_step(c, 0.0, nullptr);
        if (rc != SAC_OK) return rc;
    }
    return SAC_OK;
}

double sac3_time(const sac3_ctx* c) { return c ? c->t : 0.0; }

// FP64 diagnostics of the current state into out[kDiagVals] (synchronous)
static int diag3(sac3_ctx* c, double* out)
{
    if (!c->have_state) return fail3(c, SAC_ERR_STATE, "no state set");
    CK3(cudaSetDevice(c->p.device));
    const sac3_params& p = c->p;
    const double i12x = p.nx / (12.0 * (p.x1 - p.x0)), i12y = p.ny / (12.0 * (p.y1 - p.y0)),
                 i12z = p.nz / (12.0 * (p.z1 - p.z0));
    if (c->fp32)
        diag3_partial<float><<<kDiagBlocks, 256, 0, c->stream>>>((const float*)c->u0, c->g, i12x, i12y, i12z, c->diag);
    else
        diag3_partial<double><<<kDiagBlocks, 256, 0, c->stream>>>((const double*)c->u0, c->g, i12x, i12y, i12z, c->diag);
    CK3(cudaGetLastError());
    double* tot = c->diag + (size_t)kDiagBlocks * kDiagVals;
    diag3_final<<<1, 32, 0, c->stream>>>(c->diag, kDiagBlocks, tot);
    CK3(cudaGetLastError());
    CK3(cudaMemcpyAsync(out, tot, kDiagVals * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK3(cudaStreamSynchronize(c->stream));
    return SAC_OK;
}

int sac3_sums(sac3_ctx* c, double sums[8])
{
    if (!c || !sums) return fail3(c, SAC_ERR_ARG, "bad arguments");
    double d[kDiagVals];
    const int rc = diag3(c, d);
    if (rc != SAC_OK) return rc;
    for (int f = 0; f < NF3; ++f) sums[f] = d[f];
    return SAC_OK;
}

int sac3_divb(sac3_ctx* c, double* max_abs, double* mean_abs)
{
    if (!c) return SAC_ERR_ARG;
    double d[kDiagVals];
    const int rc = diag3(c, d);
    if (rc != SAC_OK) return rc;
    const double n = (double)c->g.nx * c->g.ny * c->g.nz;
    if (max_abs) *max_abs = d[NF3 + 1];
    if (mean_abs) *mean_abs = d[NF3] / n;
    return SAC_OK;
}

int sac3_debug_drop_copies(sac3_ctx* c, int on)
{
    if (!c) return SAC_ERR_ARG;
    if (!c->fp32) return fail3(c, SAC_ERR_ARG, "the copy-wait hook applies to FP32 contexts");
    c->drop_copies = on ? 1 : 0;
    return SAC_OK;
}

}  // extern "C"
