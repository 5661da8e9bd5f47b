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
// kernel (f3::stage3_f32), both in sac3d_f32.cu (a unit compiled with FMA
// contraction); both f3 kernels march column tiles through z fed by
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
#include "sac3d.cuh"

using namespace sac3d;

namespace {

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
        if (cf.hd) CK3(f3::launch_shock(sh, g, cf, sntx, sgrid, c->status, c->m_shk[ri], c->stream));
        // stage 4 reduces the signal speeds of the new state for the next step
        if (stage == 4) CK3(cudaMemsetAsync(c->keys, 0, 3 * sizeof(unsigned long long), c->stream));
        const f3::Maps m{c->m_full[ri], c->m_col[ri], c->m_sh_full, c->m_sh_col, c->m_col[0], c->m_acc_col};
        CK3(f3::launch_stage(stage, in, sh, u0, acc, out, g, cf, c->keys, c->status, m, c->stream));
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
static int step3(sac3_ctx* c, double dt_in, double* dt_taken, double t_end = std::numeric_limits<double>::infinity())
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
    // the last step of a run to t_end is clipped so that t lands exactly on t_end
    const bool last = c->t + dt >= t_end;
    if (last) dt = t_end - c->t;
    if (c->fp32) {
        const int rc = fused_f32(c, dt, cm, dd, dt_taken);
        if (rc == SAC_OK && last) c->t = t_end;
        return rc;
    }
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
    c->t = last ? t_end : c->t + dt;
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
    if (rc == SAC_OK && c->fp32 && f3::prepare() != cudaSuccess) rc = fail3(c, SAC_ERR_CUDA, "cudaFuncSetAttribute");
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

int sac3_run_to(sac3_ctx* c, double t_end, long max_steps, long* steps_taken)
{
    if (steps_taken) *steps_taken = 0;
    if (!c) return SAC_ERR_ARG;
    if (!c->have_state) return fail3(c, SAC_ERR_STATE, "no state set");
    if (!std::isfinite(t_end)) return fail3(c, SAC_ERR_ARG, "t_end must be finite");
    CK3(cudaSetDevice(c->p.device));
    long n = 0;
    while (c->t < t_end && (max_steps < 0 || n < max_steps)) {
        const int rc = c->fp32 ? step3<float>(c, 0.0, nullptr, t_end) : step3<double>(c, 0.0, nullptr, t_end);
        if (rc != SAC_OK) {
            if (steps_taken) *steps_taken = n;
            return rc;
        }
        ++n;
    }
    if (steps_taken) *steps_taken = n;
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
