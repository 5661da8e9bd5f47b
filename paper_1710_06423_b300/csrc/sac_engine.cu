// sac_engine.cu -- host engine and C ABI (include/sac.h) of the B300 SAC-family
// ideal-MHD step: context and device buffers, state import/export with ghost
// filling, the per-step control kernel, CUDA-graph replay of RK steps, FP64
// conservation sums and error reporting.
#include <cuda_runtime.h>
#include <math_constants.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <limits>
#include <map>
#include <mutex>
#include <tuple>

#include "../../include/sac.h"
#include "sac_internal.cuh"
#include "speed.cuh"

using namespace sac;

namespace {


__host__ __device__ inline int wrapi(int i, int n) { int r = i % n; return r < 0 ? r + n : r; }
__host__ __device__ inline int clampi(int i, int n) { return i < 0 ? 0 : (i >= n ? n - 1 : i); }

// interior index read by padded index i (ghosts included) under the
// set-up rule: periodic wraps, fixed and outflow take the nearest cell
__device__ inline int src_index(int i, int n, int bc) {
    return bc == BC_PERIODIC ? wrapi(i, n) : clampi(i, n);
}

// ---- state import / export --------------------------------------------------
// Packed [nf][ny][nx] (double or T) -> ghost-padded T, every ghost filled by
// the set-up rule (fixed sides become the held values).
template <typename T, typename S>
__global__ void import_kernel(const S* __restrict__ src, T* __restrict__ dst, Layout L, int nf,
                              int bc_x, int bc_y, bool bgfield)
{
    const long long ex = L.nx + 2 * GY, ey = L.ny + 2 * GY;
    const long long total = (long long)nf * ex * ey;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < total;
         v += (long long)gridDim.x * blockDim.x) {
        int f = (int)(v / (ex * ey));
        long long r = v - (long long)f * ex * ey;
        int j = (int)(r / ex) - GY, i = (int)(r % ex) - GY;
        int si = src_index(i, L.nx, bc_x), sj = src_index(j, L.ny, bc_y);
        dst[L.idx(f, i, j, bgfield)] = (T)src[((long long)f * L.ny + sj) * L.nx + si];
    }
}

template <typename T, typename D>
__global__ void export_kernel(const T* __restrict__ src, D* __restrict__ dst, Layout L, int nf, bool bgfield)
{
    const long long n = (long long)L.nx * L.ny, total = n * nf;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < total;
         v += (long long)gridDim.x * blockDim.x) {
        int f = (int)(v / n);
        long long r = v - (long long)f * n;
        int j = (int)(r / L.nx), i = (int)(r % L.nx);
        dst[v] = (D)src[L.idx(f, i, j, bgfield)];
    }
}

// ---- signal speed of the current state (section 2: the maximum wave speed
// sets the hyper-viscosity and the step) ---------------------------------------
template <typename T, bool BG>
__global__ void cmax_kernel(const T* __restrict__ w, const T* __restrict__ bg, Layout L, double gamma,
                            DevScalars* sc)
{
    __shared__ unsigned long long red[2][32];
    unsigned long long m[2] = {0ull, 0ull};
    const long long n = (long long)L.nx * L.ny;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n;
         v += (long long)gridDim.x * blockDim.x) {
        int j = (int)(v / L.nx), i = (int)(v % L.nx);
        T q[NF];
        for (int f = 0; f < NF; ++f) q[f] = w[L.idx(f, i, j, false)];
        T sx, sy;
        if (BG)
            signal_speeds<T, true>(q[0], q[1], q[2], q[3], q[4], q[5],
                                   bg[L.idx(0, i, j, true)], bg[L.idx(1, i, j, true)],
                                   bg[L.idx(2, i, j, true)], bg[L.idx(3, i, j, true)], (T)gamma, sx, sy);
        else
            signal_speeds<T, false>(q[0], q[1], q[2], q[3], q[4], q[5],
                                    (T)0, (T)0, (T)0, (T)0, (T)gamma, sx, sy);
        unsigned long long a = speed_key(sx), b = speed_key(sy);
        m[0] = a > m[0] ? a : m[0];
        m[1] = b > m[1] ? b : m[1];
    }
    for (int d = 0; d < 2; ++d) {
        unsigned long long x = m[d];
        for (int o = 16; o > 0; o >>= 1) {
            unsigned long long y = __shfl_xor_sync(0xffffffffu, x, o);
            x = y > x ? y : x;
        }
        if ((threadIdx.x & 31) == 0) red[d][threadIdx.x >> 5] = x;
    }
    __syncthreads();
    if (threadIdx.x < 2) {
        unsigned long long x = 0ull;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) x = red[threadIdx.x][k] > x ? red[threadIdx.x][k] : x;
        atomicMax(&sc->cmax_bits[threadIdx.x], x);
    }
}

// ---- step control -------------------------------------------------------------
__global__ void reset_kernel(DevScalars* sc, double t)
{
    sc->t = t; sc->t_end = CUDART_INF; sc->dt = 0.0; sc->fixed_dt = 0.0;
    sc->cmax_step[0] = sc->cmax_step[1] = 0.0;
    sc->cmax_bits[0] = sc->cmax_bits[1] = 0ull;
    sc->steps = 0; sc->skip = 0; sc->done = 0; sc->status = ST_OK;
}

__global__ void fixed_dt_kernel(DevScalars* sc, double dt) { sc->fixed_dt = dt > 0.0 ? dt : 0.0; }

__global__ void control_kernel(DevScalars* sc, double t_end)
{
    sc->t_end = t_end;
    sc->done = (sc->t >= t_end) ? 1 : 0;
}

// Start one RK step (see step_begin in sac_internal.cuh).
__global__ void begin_step_kernel(DevScalars* sc, double dx, double dy, double courant, int fp32,
                                  double dt_override)
{
    pdl_launch_dependents();
    pdl_wait();
    step_begin(sc, dx, dy, courant, fp32, dt_override);
}

// ---- FP64 conservation sums (deterministic two-pass) ---------------------------
template <typename T>
__global__ void sums_partial_kernel(const T* __restrict__ w, Layout L, double* __restrict__ part)
{
    __shared__ double red[NF][32];
    double acc[NF] = {0, 0, 0, 0, 0, 0};
    const long long n = (long long)L.nx * L.ny;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n;
         v += (long long)gridDim.x * blockDim.x) {
        int j = (int)(v / L.nx), i = (int)(v % L.nx);
        for (int f = 0; f < NF; ++f) acc[f] += (double)w[L.idx(f, i, j, false)];
    }
    for (int f = 0; f < NF; ++f) {
        double x = acc[f];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if ((threadIdx.x & 31) == 0) red[f][threadIdx.x >> 5] = x;
    }
    __syncthreads();
    if (threadIdx.x < NF) {
        double x = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) x += red[threadIdx.x][k];
        part[blockIdx.x * NF + threadIdx.x] = x;
    }
}

__global__ void sums_final_kernel(const double* __restrict__ part, int nb, double* __restrict__ out)
{
    if (threadIdx.x < NF) {
        double x = 0.0;
        for (int b = 0; b < nb; ++b) x += part[b * NF + threadIdx.x];
        out[threadIdx.x] = x;
    }
}

// ---- discrete divergence of the total magnetic field --------------------------
// div B = D_x Bx + D_y By with the fourth-order central difference of
// section 2 (D f = (f[-2] - 8 f[-1] + 8 f[+1] - f[+2]) / 12h), on B = B~ + B_b,
// evaluated in FP64 from the stored values.  A cell counts when its stencil
// stays inside the interior or wraps across a periodic side; a direction of
// one cell contributes no derivative.  Per block: max |div B| and sum |div B|.
// maximum that keeps a NaN (fmax would drop it): a non-finite state shows in both outputs
__device__ inline double max_nan(double a, double b) { return (a > b || a != a) ? a : b; }

__device__ inline bool divb_cell_in(int i, int n, int bc) {
    return n == 1 || bc == BC_PERIODIC || (i >= 2 && i < n - 2);
}

template <typename T, bool BG>
__global__ void divb_partial_kernel(const T* __restrict__ w, const T* __restrict__ bg, Layout L, int bc_x, int bc_y,
                                    double inv12dx, double inv12dy, double* __restrict__ part)
{
    __shared__ double red[2][32];
    double mx = 0.0, sm = 0.0;
    const long long n = (long long)L.nx * L.ny;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n;
         v += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(v / L.nx), i = (int)(v % L.nx);
        if (!divb_cell_in(i, L.nx, bc_x) || !divb_cell_in(j, L.ny, bc_y)) continue;
        auto b = [&](int f, int ii, int jj) {
            double x = (double)w[L.idx(f, ii, jj, false)];
            if (BG) x += (double)bg[L.idx(f - 2, ii, jj, true)];   // background order: rho_b, e_b, Bx_b, By_b
            return x;
        };
        double d = 0.0;
        if (L.nx > 1) {
            const int m2 = wrapi(i - 2, L.nx), m1 = wrapi(i - 1, L.nx), p1 = wrapi(i + 1, L.nx), p2 = wrapi(i + 2, L.nx);
            d += (b(4, m2, j) - 8.0 * b(4, m1, j) + 8.0 * b(4, p1, j) - b(4, p2, j)) * inv12dx;
        }
        if (L.ny > 1) {
            const int m2 = wrapi(j - 2, L.ny), m1 = wrapi(j - 1, L.ny), p1 = wrapi(j + 1, L.ny), p2 = wrapi(j + 2, L.ny);
            d += (b(5, i, m2) - 8.0 * b(5, i, m1) + 8.0 * b(5, i, p1) - b(5, i, p2)) * inv12dy;
        }
        const double a = fabs(d);
        mx = max_nan(mx, a);
        sm += a;
    }
    for (int o = 16; o > 0; o >>= 1) {
        mx = max_nan(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        sm += __shfl_xor_sync(0xffffffffu, sm, o);
    }
    if ((threadIdx.x & 31) == 0) { red[0][threadIdx.x >> 5] = mx; red[1][threadIdx.x >> 5] = sm; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, s = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) { a = max_nan(a, red[0][k]); s += red[1][k]; }
        part[2 * blockIdx.x] = a;
        part[2 * blockIdx.x + 1] = s;
    }
}

__global__ void divb_final_kernel(const double* __restrict__ part, int nb, double* __restrict__ out)
{
    if (threadIdx.x == 0) {
        double a = 0.0, s = 0.0;
        for (int b = 0; b < nb; ++b) { a = max_nan(a, part[2 * b]); s += part[2 * b + 1]; }
        out[0] = a;
        out[1] = s;
    }
}

int grid_for(long long n, int block) {
    long long g = (n + block - 1) / block;
    return (int)(g < 1 ? 1 : (g > 148 * 16 ? 148 * 16 : g));
}

// Halo strips of a block decomposition (section 3: each sub-domain exchanges
// the cells its neighbours' stencils reach).  Strip of side 0/1 (left/right):
// 3 columns over the ghost-extended height, rows -3 .. ny+2; side 2/3
// (bottom/top): 3 rows over the ghost-extended width, columns -3 .. nx+2.
// Packed [nf][rows][cols].  pack reads the interior cells next to the side,
// unpack writes the ghost cells beyond it.
struct Strip {
    int i0, j0, cols, rows;
};
__host__ __device__ inline Strip halo_strip(const Layout& L, int side, bool unpack)
{
    Strip s;
    if (side < 2) {
        s.cols = GY; s.rows = L.ny + 2 * GY; s.j0 = -GY;
        s.i0 = side == 0 ? (unpack ? -GY : 0) : (unpack ? L.nx : L.nx - GY);
    } else {
        s.cols = L.nx + 2 * GY; s.rows = GY; s.i0 = -GY;
        s.j0 = side == 2 ? (unpack ? -GY : 0) : (unpack ? L.ny : L.ny - GY);
    }
    return s;
}

template <typename T>
__global__ void halo_pack_kernel(T* __restrict__ buf, Layout L, Strip st, T* __restrict__ packed, int unpack)
{
    const long long per = (long long)st.cols * st.rows, total = per * NF;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < total; v += (long long)gridDim.x * blockDim.x) {
        const int f = (int)(v / per);
        const long long r = v - (long long)f * per;
        const int j = st.j0 + (int)(r / st.cols), i = st.i0 + (int)(r % st.cols);
        const long long e = L.idx(f, i, j, false);
        if (unpack) buf[e] = packed[v];
        else packed[v] = buf[e];
    }
}

// The running maxima as non-negative signed 64-bit keys (a reduction over
// sub-domains may then use a signed maximum): a speed key is the bit pattern of
// a non-negative float or double; a key with the top bit set (a NaN with the
// sign bit) becomes INT64_MAX, which decodes as a NaN in either precision.
__global__ void cmax_bits_copy_kernel(DevScalars* sc, unsigned long long* bits, int to_scalars)
{
    if (threadIdx.x < 2) {
        if (to_scalars) {
            sc->cmax_bits[threadIdx.x] = bits[threadIdx.x];
        } else {
            const unsigned long long k = sc->cmax_bits[threadIdx.x];
            bits[threadIdx.x] = k >> 63 ? 0x7fffffffffffffffull : k;
        }
    }
}

}  // namespace

#include "sac_ctx.h"

static const char* kStatusNames[] = {"SAC_OK", "SAC_ERR_ARG", "SAC_ERR_STATE", "SAC_ERR_CUDA",
                                     "SAC_ERR_OOM", "SAC_ERR_NONFINITE", "SAC_ERR_TIMEOUT"};

static int fail(sac_ctx* c, int code, const char* fmt, ...)
{
    if (c) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(c->err, sizeof(c->err), fmt, ap);
        va_end(ap);
    }
    return code;
}

#define CK(call)                                                                          \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return fail(c, e_ == cudaErrorMemoryAllocation ? SAC_ERR_OOM : SAC_ERR_CUDA,  \
                        "%s failed: %s", #call, cudaGetErrorString(e_));                  \
    } while (0)

static long long round_up(long long v, long long m) { return (v + m - 1) / m * m; }

// Stage input / output buffers of RK stage 1..4: ping-pong SA, SB; U0 is the
// stencil input of stage 1 and is rewritten by stage 4.
static void stage_buffers(const sac_ctx* c, int stage, void** sin, void** sout)
{
    *sin = stage == 1 ? c->u0 : (stage == 2 ? c->sa : (stage == 3 ? c->sb : c->sa));
    *sout = stage == 1 ? c->sa : (stage == 2 ? c->sb : (stage == 3 ? c->sa : c->u0));
}

template <typename T>
static void fill_stage_args(const sac_ctx* c, int stage, StageArgs<T>* a)
{
    void *sin, *sout;
    stage_buffers(c, stage, &sin, &sout);
    a->sin = (const T*)sin; a->u0 = (const T*)c->u0; a->acc = (T*)c->acc;
    a->sout = (T*)sout; a->bg = (const T*)c->bg; a->sc = c->sc; a->L = c->L;
    a->dx = c->dx; a->dy = c->dy;
    a->gamma = c->p.gamma;
    for (int f = 0; f < NF; ++f) a->c2[f] = c->p.c2[f];
    a->c_shk = c->p.c_shk; a->bc_x = c->p.bc_x; a->bc_y = c->p.bc_y;
    a->grav[0] = c->p.gravity[0]; a->grav[1] = c->p.gravity[1];
    a->hd_single_face = c->p.hd_single_face;
    a->tile = c->tile % NTILE_SHAPES;
    a->kernel_ghosts = c->tile >= NTILE_SHAPES;
    a->derive_f32();
}

void sac_fp32_stage_args(const sac_ctx* c, int stage, StageArgs<float>* out) { fill_stage_args<float>(c, stage, out); }

// Enqueue the kernel of one RK stage (1..4).
static cudaError_t enqueue_stage_one(sac_ctx* c, cudaStream_t s, int stage)
{
    const bool hd = c->p.hyperdiffusion != 0, bgp = c->p.has_background != 0;
    if (c->fp32) {
        StageArgs<float> a;
        fill_stage_args<float>(c, stage, &a);
        return launch_stage_fp32(a, stage, hd, bgp, s);
    }
    StageArgs<double> a;
    fill_stage_args<double>(c, stage, &a);
    return launch_stage_fp64(a, stage, hd, bgp, s);
}

// Enqueue the four stage kernels of one step (after begin_step).
static cudaError_t enqueue_stages(sac_ctx* c, cudaStream_t s)
{
    for (int stage = 1; stage <= 4; ++stage) {
        cudaError_t e = enqueue_stage_one(c, s, stage);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

static cudaError_t enqueue_step(sac_ctx* c, cudaStream_t s, double dt_override)
{
    const double dx = c->dx, dy = c->dy;
    // FP32: the step-control kernel and the stage kernels overlap their launches (pdl_wait)
    cudaError_t e = c->fp32 ? launch_pdl(begin_step_kernel, dim3(1), dim3(1), 0, s, c->sc, dx, dy, c->p.courant, 1,
                                         dt_override)
                            : (begin_step_kernel<<<1, 1, 0, s>>>(c->sc, dx, dy, c->p.courant, 0, dt_override),
                               cudaGetLastError());
    if (e != cudaSuccess) return e;
    return enqueue_stages(c, s);
}

static cudaError_t capture(sac_ctx* c, int nsteps, cudaGraphExec_t* out)
{
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    for (int k = 0; k < nsteps && e == cudaSuccess; ++k) e = enqueue_step(c, c->cap, 0.0);
    cudaError_t e2 = cudaStreamEndCapture(c->cap, &g);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(out, g, 0);
    if (g) cudaGraphDestroy(g);
    return e;
}

static int launch_cmax(sac_ctx* c)
{
    const int block = 256;
    long long n = (long long)c->p.nx * c->p.ny;
    int grid = grid_for(n, block);
    // the running maximum was zeroed by reset_kernel; reduce the current state into it
    if (c->fp32) {
        if (c->p.has_background)
            cmax_kernel<float, true><<<grid, block, 0, c->stream>>>((const float*)c->u0, (const float*)c->bg, c->L, c->p.gamma, c->sc);
        else
            cmax_kernel<float, false><<<grid, block, 0, c->stream>>>((const float*)c->u0, nullptr, c->L, c->p.gamma, c->sc);
    } else {
        if (c->p.has_background)
            cmax_kernel<double, true><<<grid, block, 0, c->stream>>>((const double*)c->u0, (const double*)c->bg, c->L, c->p.gamma, c->sc);
        else
            cmax_kernel<double, false><<<grid, block, 0, c->stream>>>((const double*)c->u0, nullptr, c->L, c->p.gamma, c->sc);
    }
    CK(cudaGetLastError());
    return SAC_OK;
}

// Read the device scalars (synchronises the context's stream).
static int pull_scalars(sac_ctx* c)
{
    CK(cudaMemcpyAsync(c->hsc, c->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (c->hsc->status == ST_ERR_NONFINITE)
        return fail(c, SAC_ERR_NONFINITE, "non-finite state or step after %lld steps (t = %.17g)",
                    (long long)c->hsc->steps, c->hsc->t);
    if (c->hsc->status != ST_OK)
        return fail(c, SAC_ERR_TIMEOUT, "device status %d", c->hsc->status);
    return SAC_OK;
}

static int set_t_end(sac_ctx* c, double t_end)
{
    control_kernel<<<1, 1, 0, c->stream>>>(c->sc, t_end);
    CK(cudaGetLastError());
    c->t_end_host = t_end;
    return SAC_OK;
}

static int finish_set_state(sac_ctx* c, double t)
{
    // every stage buffer carries the same ghosts (fixed sides are never rewritten)
    const size_t bytes = NF * (size_t)c->L.fstride * c->esz;
    CK(cudaMemcpyAsync(c->sa, c->u0, bytes, cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaMemcpyAsync(c->sb, c->u0, bytes, cudaMemcpyDeviceToDevice, c->stream));
    reset_kernel<<<1, 1, 0, c->stream>>>(c->sc, t);
    CK(cudaGetLastError());
    c->t_end_host = std::numeric_limits<double>::infinity();
    int rc = launch_cmax(c);
    if (rc != SAC_OK) return rc;
    c->have_state = true;
    c->last_stage = 0;
    return SAC_OK;
}

template <typename S>
static int import_fields(sac_ctx* c, const S* src, void* dst, int nf, bool background)
{
    const int block = 256;
    long long n = (long long)nf * (c->p.nx + 2 * GY) * (c->p.ny + 2 * GY);
    int bcx = c->p.bc_x, bcy = c->p.bc_y;
    if (c->fp32)
        import_kernel<float, S><<<grid_for(n, block), block, 0, c->stream>>>(src, (float*)dst, c->L, nf, bcx, bcy, background);
    else
        import_kernel<double, S><<<grid_for(n, block), block, 0, c->stream>>>(src, (double*)dst, c->L, nf, bcx, bcy, background);
    CK(cudaGetLastError());
    return SAC_OK;
}

// ============================================================================
extern "C" {

void sac_default_params(sac_params* p)
{
    if (!p) return;
    memset(p, 0, sizeof(*p));
    p->nx = 64; p->ny = 64;
    p->x0 = 0.0; p->x1 = 1.0; p->y0 = 0.0; p->y1 = 1.0;
    p->gamma = 5.0 / 3.0; p->courant = 0.3;
    p->bc_x = SAC_BC_PERIODIC; p->bc_y = SAC_BC_PERIODIC;
    p->precision = SAC_FP64;
    p->hyperdiffusion = 1;
    const double c2[6] = {0.02, 0.1, 0.1, 0.02, 0.02, 0.02};
    for (int f = 0; f < 6; ++f) p->c2[f] = c2[f];
    p->c_shk = 0.5;
    p->has_background = 0;
    p->device = 0;
    p->stream = nullptr;
}

const char* sac_status_string(int code)
{
    if (code > 0 || code < -6) return "SAC_UNKNOWN";
    return kStatusNames[-code];
}

const char* sac_last_error(const sac_ctx* c) { return c ? c->err : "no context"; }

// Tile shapes the tuner chose in this process, per run configuration (grid
// size, hyper-diffusion, background): later contexts of the same configuration
// start with that shape.
using TileKey = std::tuple<int, int, int, int>;
static std::map<TileKey, int> g_tile_cache;
static std::mutex g_tile_mu;
static TileKey tile_key(const sac_params& p) { return TileKey{p.nx, p.ny, p.hyperdiffusion, p.has_background}; }

static void drop_graphs(sac_ctx* c)
{
    if (c->g1) cudaGraphExecDestroy(c->g1);
    if (c->gN) cudaGraphExecDestroy(c->gN);
    c->g1 = c->gN = nullptr;
}

void sac_free(sac_ctx* c)
{
    if (!c) return;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(c->p.device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    drop_graphs(c);
    cudaFree(c->u0); cudaFree(c->sa); cudaFree(c->sb); cudaFree(c->acc); cudaFree(c->bg);
    cudaFree(c->sc); cudaFree(c->staging); cudaFree(c->part);
    if (c->hsc) cudaFreeHost(c->hsc);
    if (c->cap) cudaStreamDestroy(c->cap);
    cudaSetDevice(prev);
    delete c;
}

int sac_init(const sac_params* p, sac_ctx** out)
{
    if (out) *out = nullptr;
    sac_ctx* c = nullptr;
    if (!p || !out) return SAC_ERR_ARG;
    if (p->nx < 1 || p->ny < 1 || p->nx > 65536 || p->ny > 65536) return SAC_ERR_ARG;
    if (!(p->x1 > p->x0) || !(p->y1 > p->y0) || !(p->gamma > 1.0) || !(p->courant > 0.0)) return SAC_ERR_ARG;
    if (p->bc_x < 0 || p->bc_x > 2 || p->bc_y < 0 || p->bc_y > 2) return SAC_ERR_ARG;
    if (p->precision != SAC_FP64 && p->precision != SAC_FP32) return SAC_ERR_ARG;
    for (int f = 0; f < 6; ++f) if (!(p->c2[f] >= 0.0)) return SAC_ERR_ARG;
    if (!(p->c_shk >= 0.0)) return SAC_ERR_ARG;
    if (!std::isfinite(p->gravity[0]) || !std::isfinite(p->gravity[1])) return SAC_ERR_ARG;
    if ((p->gravity[0] != 0.0 || p->gravity[1] != 0.0) && !p->has_background) return SAC_ERR_ARG;
    if (p->hd_single_face != 0 && p->hd_single_face != 1) return SAC_ERR_ARG;
    if (p->hd_single_face && p->precision == SAC_FP32 &&
        (p->has_background || p->gravity[0] != 0.0 || p->gravity[1] != 0.0))
        return SAC_ERR_ARG;

    c = new sac_ctx();
    c->p = *p;
    c->dx = (p->x1 - p->x0) / p->nx;
    c->dy = (p->y1 - p->y0) / p->ny;
    c->fp32 = p->precision == SAC_FP32;
    c->esz = c->fp32 ? 4 : 8;
    c->stream = (cudaStream_t)p->stream;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || p->device < 0 || p->device >= ndev) {
        fail(c, SAC_ERR_ARG, "device %d not available", p->device);
        sac_free(c);
        return SAC_ERR_ARG;
    }
    int rc = SAC_OK;
    do {
        cudaError_t e = cudaSetDevice(p->device);
        if (e != cudaSuccess) { rc = fail(c, SAC_ERR_CUDA, "cudaSetDevice: %s", cudaGetErrorString(e)); break; }
        Layout& L = c->L;
        L.nx = p->nx; L.ny = p->ny;
        L.pitch = (int)round_up(round_up(p->nx, TILE_X_MAX) + 2 * GX, 32);
        L.rows = (int)(round_up(p->ny, TILE_Y_MAX) + 2 * GY);
        L.fstride = round_up((long long)L.pitch * L.rows, 64);
        L.paired = c->fp32 ? 1 : 0;   // FP32: three float2 planes of fstride elements each
        const size_t fbytes = (size_t)L.fstride * c->esz;
        void** bufs[4] = {&c->u0, &c->sa, &c->sb, &c->acc};
        for (int b = 0; b < 4 && rc == SAC_OK; ++b) {
            e = cudaMalloc(bufs[b], NF * fbytes);
            if (e != cudaSuccess) rc = fail(c, SAC_ERR_OOM, "cudaMalloc of %zu bytes: %s", NF * fbytes, cudaGetErrorString(e));
            else e = cudaMemset(*bufs[b], 0, NF * fbytes);
        }
        if (rc != SAC_OK) break;
        if (p->has_background) {
            e = cudaMalloc(&c->bg, NBG * fbytes);
            if (e != cudaSuccess) { rc = fail(c, SAC_ERR_OOM, "background alloc: %s", cudaGetErrorString(e)); break; }
            cudaMemset(c->bg, 0, NBG * fbytes);
        }
        if (cudaMalloc(&c->sc, sizeof(DevScalars)) != cudaSuccess ||
            cudaMallocHost(&c->hsc, sizeof(DevScalars)) != cudaSuccess ||
            cudaMalloc(&c->part, (kSumBlocks + 1) * NF * sizeof(double)) != cudaSuccess) {
            rc = fail(c, SAC_ERR_OOM, "scalar allocation failed");
            break;
        }
        e = prepare_stage_fp64();
        if (e == cudaSuccess) e = prepare_stage_fp32();
        if (e != cudaSuccess) { rc = fail(c, SAC_ERR_CUDA, "kernel set-up: %s", cudaGetErrorString(e)); break; }
        e = cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking);
        if (e != cudaSuccess) { rc = fail(c, SAC_ERR_CUDA, "stream: %s", cudaGetErrorString(e)); break; }
        e = cudaMemsetAsync(c->sc, 0, sizeof(DevScalars), c->stream);   // (drop_copies off)
        if (e != cudaSuccess) { rc = fail(c, SAC_ERR_CUDA, "init: %s", cudaGetErrorString(e)); break; }
        reset_kernel<<<1, 1, 0, c->stream>>>(c->sc, 0.0);
        e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) { rc = fail(c, SAC_ERR_CUDA, "init: %s", cudaGetErrorString(e)); break; }
        if (c->fp32) {
            std::lock_guard<std::mutex> lk(g_tile_mu);
            auto it = g_tile_cache.find(tile_key(*p));
            if (it != g_tile_cache.end()) c->tile = it->second;
        }
    } while (0);
    if (rc != SAC_OK) {
        sac_free(c);
        return rc;
    }
    *out = c;
    return SAC_OK;
}

int sac_set_state(sac_ctx* c, const double* w, const double* bg, double t)
{
    if (!c || !w) return fail(c, SAC_ERR_ARG, "null state");
    if ((bg != nullptr) != (c->p.has_background != 0))
        return fail(c, SAC_ERR_ARG, "background must be given iff has_background");
    if (!std::isfinite(t)) return fail(c, SAC_ERR_ARG, "time must be finite");
    CK(cudaSetDevice(c->p.device));
    const size_t n = (size_t)c->p.nx * c->p.ny;
    if (!c->staging) CK(cudaMalloc(&c->staging, NF * n * sizeof(double)));
    if (bg) {
        CK(cudaMemcpyAsync(c->staging, bg, NBG * n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
        int rc = import_fields<double>(c, c->staging, c->bg, NBG, true);
        if (rc != SAC_OK) return rc;
    }
    CK(cudaMemcpyAsync(c->staging, w, NF * n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    int rc = import_fields<double>(c, c->staging, c->u0, NF, false);
    if (rc != SAC_OK) return rc;
    rc = finish_set_state(c, t);
    if (rc != SAC_OK) return rc;
    CK(cudaStreamSynchronize(c->stream));
    return SAC_OK;
}

int sac_set_state_dev(sac_ctx* c, const void* w, const void* bg, double t)
{
    if (!c || !w) return fail(c, SAC_ERR_ARG, "null state");
    if ((bg != nullptr) != (c->p.has_background != 0))
        return fail(c, SAC_ERR_ARG, "background must be given iff has_background");
    if (!std::isfinite(t)) return fail(c, SAC_ERR_ARG, "time must be finite");
    CK(cudaSetDevice(c->p.device));
    int rc;
    if (c->fp32) {
        if (bg && (rc = import_fields<float>(c, (const float*)bg, c->bg, NBG, true)) != SAC_OK) return rc;
        if ((rc = import_fields<float>(c, (const float*)w, c->u0, NF, false)) != SAC_OK) return rc;
    } else {
        if (bg && (rc = import_fields<double>(c, (const double*)bg, c->bg, NBG, true)) != SAC_OK) return rc;
        if ((rc = import_fields<double>(c, (const double*)w, c->u0, NF, false)) != SAC_OK) return rc;
    }
    return finish_set_state(c, t);
}

int sac_get_state(sac_ctx* c, double* w, double* t)
{
    if (!c) return SAC_ERR_ARG;
    if (!c->have_state) return fail(c, SAC_ERR_STATE, "no state set");
    CK(cudaSetDevice(c->p.device));
    if (w) {
        const size_t n = (size_t)c->p.nx * c->p.ny;
        if (!c->staging) CK(cudaMalloc(&c->staging, NF * n * sizeof(double)));
        const int block = 256;
        int grid = grid_for((long long)NF * n, block);
        if (c->fp32)
            export_kernel<float, double><<<grid, block, 0, c->stream>>>((const float*)c->u0, c->staging, c->L, NF, false);
        else
            export_kernel<double, double><<<grid, block, 0, c->stream>>>((const double*)c->u0, c->staging, c->L, NF, false);
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(w, c->staging, NF * n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    }
    int rc = pull_scalars(c);
    if (t) *t = c->hsc->t;
    return rc;
}

int sac_get_state_dev(sac_ctx* c, void* w, double* t)
{
    if (!c) return SAC_ERR_ARG;
    if (!c->have_state) return fail(c, SAC_ERR_STATE, "no state set");
    CK(cudaSetDevice(c->p.device));
    if (w) {
        const long long n = (long long)c->p.nx * c->p.ny;
        const int block = 256;
        int grid = grid_for(NF * n, block);
        if (c->fp32)
            export_kernel<float, float><<<grid, block, 0, c->stream>>>((const float*)c->u0, (float*)w, c->L, NF, false);
        else
            export_kernel<double, double><<<grid, block, 0, c->stream>>>((const double*)c->u0, (double*)w, c->L, NF, false);
        CK(cudaGetLastError());
    }
    if (t) {
        int rc = pull_scalars(c);
        *t = c->hsc->t;
        return rc;
    }
    return SAC_OK;
}

int sac_step(sac_ctx* c, double dt, double* dt_taken)
{
    if (!c) return SAC_ERR_ARG;
    if (!c->have_state) return fail(c, SAC_ERR_STATE, "step before set_state");
    if (c->last_stage != 0 && c->last_stage != 4) return fail(c, SAC_ERR_STATE, "a step is half done (sac_stage)");
    if (!(dt <= 0.0) && !std::isfinite(dt)) return fail(c, SAC_ERR_ARG, "dt must be finite");
    CK(cudaSetDevice(c->p.device));
    int rc = set_t_end(c, std::numeric_limits<double>::infinity());
    if (rc != SAC_OK) return rc;
    CK(enqueue_step(c, c->stream, dt > 0.0 ? dt : 0.0));
    rc = pull_scalars(c);
    if (dt_taken) *dt_taken = c->hsc->dt;
    return rc;
}

int sac_steps(sac_ctx* c, long nsteps)
{
    if (!c) return SAC_ERR_ARG;
    if (!c->have_state) return fail(c, SAC_ERR_STATE, "step before set_state");
    if (c->last_stage != 0 && c->last_stage != 4) return fail(c, SAC_ERR_STATE, "a step is half done (sac_stage)");
    if (nsteps < 0) return fail(c, SAC_ERR_ARG, "nsteps < 0");
    CK(cudaSetDevice(c->p.device));
    if (c->t_end_host != std::numeric_limits<double>::infinity()) {
        int rc = set_t_end(c, std::numeric_limits<double>::infinity());
        if (rc != SAC_OK) return rc;
    }
    // both step graphs are captured by the first call, whatever its step count, so
    // that a later, longer call does not pay the capture (a one-time set-up)
    if (!c->g1) CK(capture(c, 1, &c->g1));
    if (!c->gN) CK(capture(c, kChunk, &c->gN));
    long left = nsteps;
    while (left >= kChunk) { CK(cudaGraphLaunch(c->gN, c->stream)); left -= kChunk; }
    while (left > 0) { CK(cudaGraphLaunch(c->g1, c->stream)); --left; }
    return SAC_OK;
}

int sac_run_to(sac_ctx* c, double t_end, long max_steps, long* steps_taken)
{
    if (steps_taken) *steps_taken = 0;
    if (!c) return SAC_ERR_ARG;
    if (!c->have_state) return fail(c, SAC_ERR_STATE, "run before set_state");
    if (c->last_stage != 0 && c->last_stage != 4) return fail(c, SAC_ERR_STATE, "a step is half done (sac_stage)");
    if (!std::isfinite(t_end)) return fail(c, SAC_ERR_ARG, "t_end must be finite");
    CK(cudaSetDevice(c->p.device));
    int rc = pull_scalars(c);
    if (rc != SAC_OK) return rc;
    const long long s0 = c->hsc->steps;
    rc = set_t_end(c, t_end);
    if (rc != SAC_OK) return rc;
    if (!c->g1) CK(capture(c, 1, &c->g1));
    if (!c->gN) CK(capture(c, kChunk, &c->gN));
    long launched = 0;
    double t = c->hsc->t, dt_last = c->hsc->dt;
    while ((max_steps < 0 || launched < max_steps) && t < t_end) {
        // enqueue about as many steps as remain (steps past t_end are skipped on the device)
        long want = 1;
        if (dt_last > 0.0) {
            double est = (t_end - t) / dt_last;
            want = est > 4096.0 ? 4096 : (long)est + 1;
        }
        if (max_steps >= 0 && want > max_steps - launched) want = max_steps - launched;
        long n = 0;
        while (want - n >= kChunk) { CK(cudaGraphLaunch(c->gN, c->stream)); n += kChunk; }
        while (n < want) { CK(cudaGraphLaunch(c->g1, c->stream)); ++n; }
        launched += n;
        rc = pull_scalars(c);
        if (rc != SAC_OK) break;
        t = c->hsc->t;
        dt_last = c->hsc->dt;
        if (c->hsc->done) break;
    }
    if (steps_taken) *steps_taken = (long)(c->hsc->steps - s0);
    return rc;
}

int sac_set_fixed_dt(sac_ctx* c, double dt)
{
    if (!c) return SAC_ERR_ARG;
    if (!(dt <= 0.0) && !std::isfinite(dt)) return fail(c, SAC_ERR_ARG, "dt must be finite");
    CK(cudaSetDevice(c->p.device));
    fixed_dt_kernel<<<1, 1, 0, c->stream>>>(c->sc, dt);
    CK(cudaGetLastError());
    return SAC_OK;
}

int sac_dt(sac_ctx* c, double* dt)
{
    if (!c || !dt) return SAC_ERR_ARG;
    if (!c->have_state) return fail(c, SAC_ERR_STATE, "no state set");
    double cx, cy;
    int rc = sac_cmax(c, &cx, &cy);
    if (rc != SAC_OK) return rc;
    const double dx = c->dx, dy = c->dy;
    double tx = dx / cx, ty = dy / cy;
    *dt = c->p.courant * std::fmin(tx, ty);
    return SAC_OK;
}

int sac_time(sac_ctx* c, double* t, long* steps)
{
    if (!c) return SAC_ERR_ARG;
    CK(cudaSetDevice(c->p.device));
    int rc = pull_scalars(c);
    if (t) *t = c->hsc->t;
    if (steps) *steps = (long)c->hsc->steps;
    return rc;
}

int sac_cmax(sac_ctx* c, double* cx, double* cy)
{
    if (!c) return SAC_ERR_ARG;
    if (!c->have_state) return fail(c, SAC_ERR_STATE, "no state set");
    CK(cudaSetDevice(c->p.device));
    int rc = pull_scalars(c);
    if (rc != SAC_OK) return rc;
    unsigned long long b[2] = {c->hsc->cmax_bits[0], c->hsc->cmax_bits[1]};
    double v[2];
    for (int d = 0; d < 2; ++d) {
        if (c->fp32) { unsigned u = (unsigned)b[d]; float f; memcpy(&f, &u, 4); v[d] = f; }
        else memcpy(&v[d], &b[d], 8);
    }
    if (cx) *cx = v[0];
    if (cy) *cy = v[1];
    return SAC_OK;
}

int sac_sums(sac_ctx* c, double sums[6])
{
    if (!c || !sums) return SAC_ERR_ARG;
    if (!c->have_state) return fail(c, SAC_ERR_STATE, "no state set");
    CK(cudaSetDevice(c->p.device));
    if (c->fp32)
        sums_partial_kernel<float><<<kSumBlocks, 256, 0, c->stream>>>((const float*)c->u0, c->L, c->part);
    else
        sums_partial_kernel<double><<<kSumBlocks, 256, 0, c->stream>>>((const double*)c->u0, c->L, c->part);
    CK(cudaGetLastError());
    sums_final_kernel<<<1, 32, 0, c->stream>>>(c->part, kSumBlocks, c->part + kSumBlocks * NF);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(sums, c->part + kSumBlocks * NF, NF * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    return pull_scalars(c);
}

int sac_divb(sac_ctx* c, double* max_abs, double* mean_abs, long long* ncells)
{
    if (!c) return SAC_ERR_ARG;
    if (!c->have_state) return fail(c, SAC_ERR_STATE, "no state set");
    CK(cudaSetDevice(c->p.device));
    const double inv12dx = c->cell_override ? 1.0 / (12.0 * c->dx) : c->p.nx / (12.0 * (c->p.x1 - c->p.x0));
    const double inv12dy = c->cell_override ? 1.0 / (12.0 * c->dy) : c->p.ny / (12.0 * (c->p.y1 - c->p.y0));
    const int bx = c->p.bc_x, by = c->p.bc_y;
    // part holds (kSumBlocks + 1) * NF doubles; this needs 2 * kSumBlocks + 2
    double* out = c->part + 2 * kSumBlocks;
    if (c->fp32) {
        if (c->p.has_background)
            divb_partial_kernel<float, true><<<kSumBlocks, 256, 0, c->stream>>>(
                (const float*)c->u0, (const float*)c->bg, c->L, bx, by, inv12dx, inv12dy, c->part);
        else
            divb_partial_kernel<float, false><<<kSumBlocks, 256, 0, c->stream>>>(
                (const float*)c->u0, nullptr, c->L, bx, by, inv12dx, inv12dy, c->part);
    } else {
        if (c->p.has_background)
            divb_partial_kernel<double, true><<<kSumBlocks, 256, 0, c->stream>>>(
                (const double*)c->u0, (const double*)c->bg, c->L, bx, by, inv12dx, inv12dy, c->part);
        else
            divb_partial_kernel<double, false><<<kSumBlocks, 256, 0, c->stream>>>(
                (const double*)c->u0, nullptr, c->L, bx, by, inv12dx, inv12dy, c->part);
    }
    CK(cudaGetLastError());
    divb_final_kernel<<<1, 32, 0, c->stream>>>(c->part, kSumBlocks, out);
    CK(cudaGetLastError());
    double h[2];
    CK(cudaMemcpyAsync(h, out, sizeof h, cudaMemcpyDeviceToHost, c->stream));
    const int rc = pull_scalars(c);
    if (rc != SAC_OK) return rc;
    auto count = [](int n, int bc) -> long long { return (n == 1 || bc == BC_PERIODIC) ? n : (n > 4 ? n - 4 : 0); };
    const long long nc = count(c->p.nx, bx) * count(c->p.ny, by);
    if (max_abs) *max_abs = h[0];
    if (mean_abs) *mean_abs = nc > 0 ? h[1] / (double)nc : 0.0;
    if (ncells) *ncells = nc;
    return SAC_OK;
}

int sac_profile_stages(sac_ctx* c, int nsteps, double ms[5])
{
    if (!c || !ms || nsteps < 1) return fail(c, SAC_ERR_ARG, "bad arguments");
    if (!c->have_state) return fail(c, SAC_ERR_STATE, "no state set");
    CK(cudaSetDevice(c->p.device));
    int rc = set_t_end(c, std::numeric_limits<double>::infinity());
    if (rc != SAC_OK) return rc;
    cudaEvent_t ev[6];
    for (int k = 0; k < 6; ++k) CK(cudaEventCreate(&ev[k]));
    double acc[5] = {0, 0, 0, 0, 0};
    const double dx = c->dx, dy = c->dy;
    for (int it = 0; it < nsteps && rc == SAC_OK; ++it) {
        cudaEventRecord(ev[0], c->stream);
        begin_step_kernel<<<1, 1, 0, c->stream>>>(c->sc, dx, dy, c->p.courant, c->fp32 ? 1 : 0, 0.0);
        cudaEventRecord(ev[1], c->stream);
        for (int stage = 1; stage <= 4; ++stage) {
            cudaError_t e = enqueue_stage_one(c, c->stream, stage);
            if (e != cudaSuccess) { rc = fail(c, SAC_ERR_CUDA, "stage launch: %s", cudaGetErrorString(e)); break; }
            cudaEventRecord(ev[1 + stage], c->stream);
        }
        if (rc != SAC_OK) break;
        cudaError_t e = cudaEventSynchronize(ev[5]);
        if (e != cudaSuccess) { rc = fail(c, SAC_ERR_CUDA, "profile: %s", cudaGetErrorString(e)); break; }
        for (int k = 0; k < 5; ++k) {
            float m = 0.f;
            cudaEventElapsedTime(&m, ev[k], ev[k + 1]);
            acc[k] += m;
        }
    }
    for (int k = 0; k < 6; ++k) cudaEventDestroy(ev[k]);
    for (int k = 0; k < 5; ++k) ms[k] = acc[k] / nsteps;
    if (rc != SAC_OK) return rc;
    return pull_scalars(c);
}

int sac_sync(sac_ctx* c)
{
    if (!c) return SAC_ERR_ARG;
    CK(cudaSetDevice(c->p.device));
    return pull_scalars(c);
}

int sac_set_tile(sac_ctx* c, int tile)
{
    if (!c) return SAC_ERR_ARG;
    if (tile < 0 || tile >= NTILE_CONFIGS) return fail(c, SAC_ERR_ARG, "unknown tile configuration %d", tile);
    if (!c->fp32) return fail(c, SAC_ERR_ARG, "tile shapes apply to FP32 contexts");
    if (tile != c->tile) {
        CK(cudaSetDevice(c->p.device));
        CK(cudaStreamSynchronize(c->stream));
        drop_graphs(c);   // the step graphs hold launches of the old shape
        c->tile = tile;
    }
    return SAC_OK;
}

int sac_get_tile(const sac_ctx* c, int* tile)
{
    if (!c || !tile) return SAC_ERR_ARG;
    *tile = c->tile;
    return SAC_OK;
}

int sac_tune(sac_ctx* c, int trials, int* tile_out, double* ms_out)
{
    if (!c) return SAC_ERR_ARG;
    if (!c->fp32) return fail(c, SAC_ERR_ARG, "tile shapes apply to FP32 contexts");
    if (trials < 1) return fail(c, SAC_ERR_ARG, "trials < 1");
    if (!c->have_state) return fail(c, SAC_ERR_STATE, "no state set");
    CK(cudaSetDevice(c->p.device));
    int rc = pull_scalars(c);
    if (rc != SAC_OK) return rc;
    rc = set_t_end(c, std::numeric_limits<double>::infinity());
    if (rc != SAC_OK) return rc;
    // snapshot of the state (with its ghosts) and of the step scalars; the
    // trials advance them and are undone afterwards
    const size_t bytes = NF * (size_t)c->L.fstride * c->esz;
    void* snap = nullptr;
    if (cudaMalloc(&snap, bytes) != cudaSuccess) return fail(c, SAC_ERR_OOM, "tuner snapshot of %zu bytes", bytes);
    DevScalars hs;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMemcpyAsync(snap, c->u0, bytes, cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hs, c->sc, sizeof hs, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    const int keep = c->tile;
    double best = 1e300;
    int bi = keep;
    // the in-kernel ghost frame exists for the plain kernels only (no background,
    // gravity or single-face variant), which otherwise ignore it
    const int nconf = c->p.has_background || c->p.hd_single_face ? (int)NTILE_SHAPES : (int)NTILE_CONFIGS;
    for (int t = 0; t < nconf && e == cudaSuccess; ++t) {
        c->tile = t;
        e = enqueue_step(c, c->stream, 0.0);                   // warm-up (tensor maps, caches)
        if (e == cudaSuccess) e = cudaEventRecord(e0, c->stream);
        for (int k = 0; k < trials && e == cudaSuccess; ++k) e = enqueue_step(c, c->stream, 0.0);
        if (e == cudaSuccess) e = cudaEventRecord(e1, c->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && ms / trials < best) { best = ms / trials; bi = t; }
        // back to the snapshot before the next shape
        if (e == cudaSuccess) e = cudaMemcpyAsync(c->u0, snap, bytes, cudaMemcpyDeviceToDevice, c->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(c->sc, &hs, sizeof hs, cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaStreamSynchronize(c->stream);
    cudaFree(snap);
    c->tile = keep;
    if (e != cudaSuccess) return fail(c, SAC_ERR_CUDA, "tuner: %s", cudaGetErrorString(e));
    rc = pull_scalars(c);   // a trial that failed on the device is reported, the state is restored
    if (rc != SAC_OK) return rc;
    rc = sac_set_tile(c, bi);
    if (rc != SAC_OK) return rc;
    {
        std::lock_guard<std::mutex> lk(g_tile_mu);
        g_tile_cache[tile_key(c->p)] = bi;
    }
    if (tile_out) *tile_out = bi;
    if (ms_out) *ms_out = best;
    return SAC_OK;
}

int sac_set_cell_size(sac_ctx* c, double dx, double dy)
{
    if (!c) return SAC_ERR_ARG;
    if (!(dx > 0.0) || !(dy > 0.0) || !std::isfinite(dx) || !std::isfinite(dy))
        return fail(c, SAC_ERR_ARG, "cell size must be finite and positive");
    CK(cudaSetDevice(c->p.device));
    CK(cudaStreamSynchronize(c->stream));
    drop_graphs(c);   // the step graphs hold the old cell size
    c->dx = dx; c->dy = dy;
    c->cell_override = true;
    return SAC_OK;
}

int sac_stage(sac_ctx* c, int stage)
{
    if (!c) return SAC_ERR_ARG;
    if (stage < 1 || stage > 4) return fail(c, SAC_ERR_ARG, "stage %d is not 1..4", stage);
    if (!c->have_state) return fail(c, SAC_ERR_STATE, "stage before set_state");
    const bool in_order = stage == 1 ? (c->last_stage == 0 || c->last_stage == 4) : c->last_stage == stage - 1;
    if (!in_order) return fail(c, SAC_ERR_STATE, "stage %d after stage %d", stage, c->last_stage);
    CK(cudaSetDevice(c->p.device));
    if (stage == 1) {
        if (c->t_end_host != std::numeric_limits<double>::infinity()) {
            int rc = set_t_end(c, std::numeric_limits<double>::infinity());
            if (rc != SAC_OK) return rc;
        }
        const double dx = c->dx, dy = c->dy;
        begin_step_kernel<<<1, 1, 0, c->stream>>>(c->sc, dx, dy, c->p.courant, c->fp32 ? 1 : 0, 0.0);
        CK(cudaGetLastError());
    }
    CK(enqueue_stage_one(c, c->stream, stage));
    c->last_stage = stage;
    return SAC_OK;
}

static int halo_args(sac_ctx* c, int side, long long* n)
{
    if (!c) return SAC_ERR_ARG;
    if (side < 0 || side > 3) return fail(c, SAC_ERR_ARG, "side %d is not 0..3", side);
    if ((side < 2 ? c->p.nx : c->p.ny) < GY) return fail(c, SAC_ERR_ARG, "a halo strip needs 3 interior cells across");
    const Strip st = halo_strip(c->L, side, false);
    *n = (long long)NF * st.cols * st.rows;
    return SAC_OK;
}

int sac_halo_size(sac_ctx* c, int side, long long* n)
{
    long long k = 0;
    int rc = halo_args(c, side, &k);
    if (rc == SAC_OK && n) *n = k;
    return rc;
}

static int halo_copy(sac_ctx* c, int side, void* buf, int unpack)
{
    long long n = 0;
    int rc = halo_args(c, side, &n);
    if (rc != SAC_OK) return rc;
    if (!buf) return fail(c, SAC_ERR_ARG, "null strip buffer");
    if (!c->have_state) return fail(c, SAC_ERR_STATE, "no state set");
    CK(cudaSetDevice(c->p.device));
    void *sin, *sout;
    stage_buffers(c, c->last_stage == 0 ? 4 : c->last_stage, &sin, &sout);   // stage 4 writes U0
    const Strip st = halo_strip(c->L, side, unpack != 0);
    const int grid = grid_for(n, 256);
    if (c->fp32)
        halo_pack_kernel<float><<<grid, 256, 0, c->stream>>>((float*)sout, c->L, st, (float*)buf, unpack);
    else
        halo_pack_kernel<double><<<grid, 256, 0, c->stream>>>((double*)sout, c->L, st, (double*)buf, unpack);
    CK(cudaGetLastError());
    return SAC_OK;
}

int sac_halo_pack(sac_ctx* c, int side, void* strip_dev) { return halo_copy(c, side, strip_dev, 0); }
int sac_halo_unpack(sac_ctx* c, int side, const void* strip_dev) { return halo_copy(c, side, (void*)strip_dev, 1); }

static int cmax_bits_copy(sac_ctx* c, void* bits, int to_scalars)
{
    if (!c || !bits) return SAC_ERR_ARG;
    if (!c->have_state) return fail(c, SAC_ERR_STATE, "no state set");
    CK(cudaSetDevice(c->p.device));
    cmax_bits_copy_kernel<<<1, 32, 0, c->stream>>>(c->sc, (unsigned long long*)bits, to_scalars);
    CK(cudaGetLastError());
    return SAC_OK;
}

int sac_get_cmax_bits(sac_ctx* c, void* bits_dev) { return cmax_bits_copy(c, bits_dev, 0); }
int sac_set_cmax_bits(sac_ctx* c, const void* bits_dev) { return cmax_bits_copy(c, (void*)bits_dev, 1); }

int sac_debug_drop_copies(sac_ctx* c, int on)
{
    if (!c) return SAC_ERR_ARG;
    if (c->p.precision != SAC_FP32) return fail(c, SAC_ERR_ARG, "the copy-wait hook applies to FP32 contexts");
    CK(cudaSetDevice(c->p.device));
    const int v = on ? 1 : 0;
    CK(cudaMemcpyAsync(&c->sc->drop_copies, &v, sizeof v, cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return SAC_OK;
}

}  // extern "C"
