// sac3d.cu -- the 3D form of the split ideal-MHD RK4 step (section 2 of
// arXiv 1710.06423 written for three-component vectors): eight conserved
// fields rho, m_x, m_y, m_z, e, B_x, B_y, B_z on a periodic box, no background.
//
// Each RK stage runs four kernels that follow the method's own order of
// operations (FP64 agrees with the FP64 3D oracle to rounding order; the unit
// is compiled without FMA contraction):
//   ghosts3   periodic ghost frame (width 3) of the stage input;
//   flux3     per ghost-extended cell: velocities and the fluxes of all eight
//             fields along x, y and z (global scratch);
//   shock3    s = max(0, -((D_x v_x + D_y v_y) + D_z v_z)) on the cells the
//             face coefficients need;
//   update3   per interior cell: k = ((H_x + H_y) + H_z) - ((D_x F_x + D_y F_y)
//             + D_z F_z) (hyper-diffusion with the maxima over three faces,
//             fourth-order flux differences) and the classical RK4 register
//             update (K = k1 + 2 k2 + 2 k3, U = U0 + dt/6 (K + k4)).
// The step's signal speeds come from one reduction over the state (ordered
// bits, NaN propagates); dt = C min(min(dx/cx, dy/cy), dz/cz) is formed on
// the host in FP64.  This first 3D path keeps the fluxes in global memory (a
// correctness-first layout: about twice the bytes of a fused tile kernel).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <limits>
#include <string>

#include "../../include/sac.h"

namespace {

constexpr int NF3 = 8;   // rho, m_x, m_y, m_z, e, B_x, B_y, B_z
constexpr int G3 = 3;    // ghost width

struct Grid3 {
    int nx, ny, nz;
    long long ex, ey, ez;   // ghost-extended extents
    long long ne;           // cells per extended field
    __host__ __device__ long long at(int i, int j, int k) const
    {
        return ((long long)(k + G3) * ey + (j + G3)) * ex + (i + G3);
    }
};

__device__ __forceinline__ int wrapn(int i, int n) { int r = i % n; return r < 0 ? r + n : r; }

template <typename T>
__global__ void ghosts3(T* __restrict__ s, Grid3 g)
{
    const long long tot = g.ne * NF3;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
        const int f = (int)(t / g.ne);
        const long long c = t - (long long)f * g.ne;
        const int i = (int)(c % g.ex) - G3, j = (int)((c / g.ex) % g.ey) - G3, k = (int)(c / (g.ex * g.ey)) - G3;
        if (i >= 0 && i < g.nx && j >= 0 && j < g.ny && k >= 0 && k < g.nz) continue;
        T* u = s + (long long)f * g.ne;
        u[c] = u[g.at(wrapn(i, g.nx), wrapn(j, g.ny), wrapn(k, g.nz))];
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

template <typename T>
__global__ void cmax3_kernel(const T* __restrict__ s, Grid3 g, T gamma, unsigned long long* __restrict__ keys)
{
    const long long n = (long long)g.nx * g.ny * g.nz, ne = g.ne;
    double mxs[3] = {0.0, 0.0, 0.0};
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(t % g.nx), j = (int)((t / g.nx) % g.ny), k = (int)(t / ((long long)g.nx * g.ny));
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
    double t = 0.0;
    bool have_state = false;
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

template <typename T>
static int step3(sac3_ctx* c, double dt_in, double* dt_taken)
{
    const Grid3& g = c->g;
    const long long n = (long long)g.nx * g.ny * g.nz;
    const double dd[3] = {(c->p.x1 - c->p.x0) / g.nx, (c->p.y1 - c->p.y0) / g.ny, (c->p.z1 - c->p.z0) / g.nz};
    // signal speeds of the step-start state (all four stages use them)
    CK3(cudaMemsetAsync(c->keys, 0, 3 * sizeof(unsigned long long), c->stream));
    cmax3_kernel<T><<<grid_for(n), 256, 0, c->stream>>>((const T*)c->u0, g, (T)c->p.gamma, c->keys);
    CK3(cudaGetLastError());
    unsigned long long hk[3];
    CK3(cudaMemcpyAsync(hk, c->keys, sizeof hk, cudaMemcpyDeviceToHost, c->stream));
    CK3(cudaStreamSynchronize(c->stream));
    double cm[3];
    for (int d = 0; d < 3; ++d) { long long b; memcpy(&b, &hk[d], 8); double x; memcpy(&x, &b, 8); cm[d] = x; }
    double dt = dt_in > 0.0 ? dt_in : c->p.courant * fmin(fmin(dd[0] / cm[0], dd[1] / cm[1]), dd[2] / cm[2]);
    if (!(dt > 0.0) || !std::isfinite(dt) || !std::isfinite(cm[0]) || !std::isfinite(cm[1]) || !std::isfinite(cm[2]))
        return fail3(c, SAC_ERR_NONFINITE, "non-finite state or step at t = %g", c->t);
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
        ghosts3<T><<<grid_for(g.ne * NF3), 256, 0, c->stream>>>(in, g);
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
    cudaFree(c->wbuf); cudaFree(c->keys);
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
    g.ex = p->nx + 2 * G3; g.ey = p->ny + 2 * G3; g.ez = p->nz + 2 * G3;
    g.ne = g.ex * g.ey * g.ez;
    const long long n = (long long)p->nx * p->ny * p->nz;
    int rc = SAC_OK;
    if (cudaSetDevice(p->device) != cudaSuccess) rc = fail3(c, SAC_ERR_CUDA, "cudaSetDevice");
    const size_t fb = (size_t)g.ne * c->esz;
    if (rc == SAC_OK &&
        (cudaMalloc(&c->u0, NF3 * fb) != cudaSuccess || cudaMalloc(&c->sa, NF3 * fb) != cudaSuccess ||
         cudaMalloc(&c->sb, NF3 * fb) != cudaSuccess ||
         cudaMalloc(&c->acc, NF3 * fb) != cudaSuccess || cudaMalloc(&c->v, 3 * fb) != cudaSuccess ||
         cudaMalloc(&c->fl, 3 * NF3 * fb) != cudaSuccess || cudaMalloc(&c->sh, fb) != cudaSuccess ||
         cudaMalloc(&c->wbuf, (size_t)NF3 * n * sizeof(double)) != cudaSuccess ||
         cudaMalloc(&c->keys, 3 * sizeof(unsigned long long)) != cudaSuccess)) {
        cudaGetLastError();
        rc = fail3(c, SAC_ERR_OOM, "device allocation failed");
    }
    if (rc == SAC_OK && (cudaMemset(c->u0, 0, NF3 * fb) != cudaSuccess || cudaMemset(c->sa, 0, NF3 * fb) != cudaSuccess ||
                         cudaMemset(c->sb, 0, NF3 * fb) != cudaSuccess || cudaMemset(c->sh, 0, fb) != cudaSuccess))
        rc = fail3(c, SAC_ERR_CUDA, "cudaMemset");
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

}  // extern "C"
