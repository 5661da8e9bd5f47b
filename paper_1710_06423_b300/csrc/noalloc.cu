// noalloc.cu -- one FP32 RK4 step on caller-owned device buffers that
// allocates nothing: its working memory (the ghost-padded RK registers and the
// step scalars) is a fixed, file-scope device array that every GPU loading the
// library holds until the process exits.
#include <cuda_runtime.h>
#include <math_constants.h>

#include <cmath>
#include <mutex>

#include "../../include/sac.h"
#include "sac_internal.cuh"
#include "speed.cuh"

using namespace sac;

namespace {

// Working memory: 256 bytes of step scalars, then four RK registers (state,
// two stage inputs, increment), each three float2 planes of kPlane elements.
// kPlane is the padded plane of a 256 x 256 grid; any grid whose padded plane
// (the same padding as sac_init) fits is accepted.
constexpr long long kPlane = 75456;
constexpr size_t kScalarBytes = 256;
constexpr size_t kRegisterBytes = 3 * (size_t)kPlane * sizeof(float2);
constexpr size_t kScratchBytes = kScalarBytes + 4 * kRegisterBytes;   // 7,244,032 bytes
static_assert(kScratchBytes == 7244032, "the header states this size");
static_assert(sizeof(DevScalars) <= kScalarBytes, "scalars must fit their slot");

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
unsigned char* g_scratch_addr[kMaxDevices] = {nullptr};   // device address of g_scratch, per device
std::mutex g_setup_mutex;                                 // guards the per-device set-up below

// Once per device, with that device current: look up the device address of the
// file-scope array (its host-side name is only a stand-in) and set the stage
// kernels' attributes.  Two host threads making their first call at the same
// time serialise here; a failed look-up is retried by the next call.
unsigned char* scratch_base(int device)
{
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    unsigned char*& base = g_scratch_addr[device];
    if (!base) {
        void* addr = nullptr;
        if (cudaGetSymbolAddress(&addr, g_scratch) != cudaSuccess || !addr) return nullptr;
        if (prepare_stage_fp32() != cudaSuccess) return nullptr;
        base = static_cast<unsigned char*>(addr);
    }
    return base;
}

long long round_up(long long v, long long m) { return (v + m - 1) / m * m; }
__device__ inline int wrap_n(int i, int n) { int r = i % n; return r < 0 ? r + n : r; }
__device__ inline int clamp_n(int i, int n) { return i < 0 ? 0 : (i >= n ? n - 1 : i); }

// Packed float [6][ny][nx] -> paired ghost-padded planes of U0, SA and SB, every
// ghost filled by the set-up rule (periodic wraps, fixed/outflow take the nearest
// interior cell); also resets the step scalars and arms the signal-speed maximum.
__global__ void na_import(const float* __restrict__ src, float* u0, float* sa, float* sb, Layout L,
                          int bc_x, int bc_y, DevScalars* sc)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        sc->t = 0.0; sc->t_end = CUDART_INF; sc->dt = 0.0; sc->fixed_dt = 0.0;
        sc->cmax_step[0] = sc->cmax_step[1] = 0.0;
        sc->cmax_bits[0] = sc->cmax_bits[1] = 0ull;
        sc->steps = 0; sc->skip = 0; sc->done = 0; sc->status = ST_OK; sc->drop_copies = 0;
    }
    const long long ex = L.nx + 2 * GY, ey = L.ny + 2 * GY, total = (long long)NF * ex * ey;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < total;
         v += (long long)gridDim.x * blockDim.x) {
        const int f = (int)(v / (ex * ey));
        const long long r = v - (long long)f * ex * ey;
        const int j = (int)(r / ex) - GY, i = (int)(r % ex) - GY;
        const int si = bc_x == BC_PERIODIC ? wrap_n(i, L.nx) : clamp_n(i, L.nx);
        const int sj = bc_y == BC_PERIODIC ? wrap_n(j, L.ny) : clamp_n(j, L.ny);
        const float x = src[((long long)f * L.ny + sj) * L.nx + si];
        const long long d = L.idx(f, i, j, false);
        u0[d] = x; sa[d] = x; sb[d] = x;
    }
}

__global__ void na_cmax(const float* __restrict__ w, Layout L, double gamma, DevScalars* sc)
{
    __shared__ unsigned long long red[2][32];
    unsigned long long m[2] = {0ull, 0ull};
    const long long n = (long long)L.nx * L.ny;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n;
         v += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(v / L.nx), i = (int)(v % L.nx);
        float q[NF];
        for (int f = 0; f < NF; ++f) q[f] = w[L.idx(f, i, j, false)];
        float sx, sy;
        signal_speeds<float, false>(q[0], q[1], q[2], q[3], q[4], q[5], 0.f, 0.f, 0.f, 0.f, (float)gamma, sx, sy);
        const unsigned long long a = speed_key(sx), b = speed_key(sy);
        m[0] = a > m[0] ? a : m[0];
        m[1] = b > m[1] ? b : m[1];
    }
    for (int d = 0; d < 2; ++d) {
        unsigned long long x = m[d];
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long y = __shfl_xor_sync(0xffffffffu, x, o);
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

__global__ void na_begin(DevScalars* sc, double dx, double dy, double courant, double dt_override)
{
    step_begin(sc, dx, dy, courant, 1, dt_override);
}

__global__ void na_export(const float* __restrict__ u0, float* __restrict__ dst, Layout L)
{
    const long long n = (long long)L.nx * L.ny, total = n * NF;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < total;
         v += (long long)gridDim.x * blockDim.x) {
        const int f = (int)(v / n);
        const long long r = v - (long long)f * n;
        const int j = (int)(r / L.nx), i = (int)(r % L.nx);
        dst[v] = u0[L.idx(f, i, j, false)];
    }
}

int grid_for(long long n) {
    const long long g = (n + 255) / 256;
    return (int)(g < 1 ? 1 : (g > 148 * 16 ? 148 * 16 : g));
}

}  // namespace

extern "C" int sac_step_noalloc(const sac_params* p, const float* w_in, float* w_out, double dt, double* dt_taken)
{
    if (!p || !w_in || !w_out) return SAC_ERR_ARG;
    if (p->precision != SAC_FP32 || p->has_background) return SAC_ERR_ARG;
    if (p->gravity[0] != 0.0 || p->gravity[1] != 0.0 || p->hd_single_face) return SAC_ERR_ARG;
    if (p->nx < 1 || p->ny < 1 || p->nx > 65536 || p->ny > 65536) return SAC_ERR_ARG;
    if (!(p->x1 > p->x0) || !(p->y1 > p->y0) || !(p->gamma > 1.0) || !(p->courant > 0.0)) return SAC_ERR_ARG;
    if (p->bc_x < 0 || p->bc_x > 2 || p->bc_y < 0 || p->bc_y > 2) return SAC_ERR_ARG;
    if (!(dt <= 0.0) && !std::isfinite(dt)) return SAC_ERR_ARG;
    if (p->device < 0 || p->device >= kMaxDevices) return SAC_ERR_ARG;

    // the padded layout sac_init would use; it must fit the fixed working memory
    Layout L;
    L.nx = p->nx; L.ny = p->ny;
    L.pitch = (int)round_up(round_up(p->nx, TILE_X_MAX) + 2 * GX, 32);
    L.rows = (int)(round_up(p->ny, TILE_Y_MAX) + 2 * GY);
    L.fstride = round_up((long long)L.pitch * L.rows, 64);
    L.paired = 1;
    if (L.fstride > kPlane) return SAC_ERR_TOO_LARGE;

    if (cudaSetDevice(p->device) != cudaSuccess) return SAC_ERR_CUDA;
    unsigned char* base = scratch_base(p->device);
    if (!base) return SAC_ERR_CUDA;
    DevScalars* sc = reinterpret_cast<DevScalars*>(base);
    float* reg[4];
    for (int k = 0; k < 4; ++k) reg[k] = reinterpret_cast<float*>(base + kScalarBytes + k * kRegisterBytes);
    float *u0 = reg[0], *sa = reg[1], *sb = reg[2], *acc = reg[3];

    cudaStream_t s = (cudaStream_t)p->stream;
    const double dx = (p->x1 - p->x0) / p->nx, dy = (p->y1 - p->y0) / p->ny;
    na_import<<<grid_for((long long)NF * (p->nx + 2 * GY) * (p->ny + 2 * GY)), 256, 0, s>>>(
        w_in, u0, sa, sb, L, p->bc_x, p->bc_y, sc);
    na_cmax<<<grid_for((long long)p->nx * p->ny), 256, 0, s>>>(u0, L, p->gamma, sc);
    na_begin<<<1, 1, 0, s>>>(sc, dx, dy, p->courant, dt > 0.0 ? dt : 0.0);
    if (cudaGetLastError() != cudaSuccess) return SAC_ERR_CUDA;

    StageArgs<float> a;
    a.u0 = u0; a.acc = acc; a.bg = nullptr; a.sc = sc; a.L = L;
    a.dx = dx; a.dy = dy; a.gamma = p->gamma;
    for (int f = 0; f < NF; ++f) a.c2[f] = p->c2[f];
    a.c_shk = p->c_shk; a.bc_x = p->bc_x; a.bc_y = p->bc_y;
    a.grav[0] = a.grav[1] = 0.0;
    a.hd_single_face = 0;
    a.derive_f32();
    for (int stage = 1; stage <= 4; ++stage) {
        a.sin = stage == 1 ? u0 : (stage == 2 ? sa : (stage == 3 ? sb : sa));
        a.sout = stage == 1 ? sa : (stage == 2 ? sb : (stage == 3 ? sa : u0));
        if (launch_stage_fp32(a, stage, p->hyperdiffusion != 0, false, s) != cudaSuccess) return SAC_ERR_CUDA;
    }
    na_export<<<grid_for((long long)NF * p->nx * p->ny), 256, 0, s>>>(u0, w_out, L);
    if (cudaGetLastError() != cudaSuccess) return SAC_ERR_CUDA;

    if (dt_taken) {
        DevScalars h;
        if (cudaMemcpyAsync(&h, sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return SAC_ERR_CUDA;
        // as the context path reports them: a non-finite state or step, else a
        // staging wait of a stage kernel that gave up
        if (h.status == ST_ERR_NONFINITE) return SAC_ERR_NONFINITE;
        if (h.status != ST_OK) return SAC_ERR_TIMEOUT;
        *dt_taken = h.dt;
    }
    return SAC_OK;
}
