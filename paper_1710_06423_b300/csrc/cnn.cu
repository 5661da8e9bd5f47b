// cnn.cu -- the learned coarse-grid correction: a 4-layer periodic 3x3 CNN
// (8 -> 32 -> 32 -> 32 -> 6 channels, ReLU) whose output, scaled per field, is
// added to the coarse state after each RK4 step.  Forward and backward run on
// BF16 tensor cores (mma.sync m16n8k16, FP32 accumulation) in implicit-GEMM
// kernels written here; the FP32 master weights are updated with Adam.
//
// Activations are NHWC bf16 ([pixel][channel], channels padded to 16 or 32).
// Layer k weights for the forward pass are bf16 [cout][tap][cin] (tap = 3a+e,
// a the row offset, e the column offset, cin contiguous); for the input
// gradient they are bf16 [cin][tap'][cout] with tap' = 8 - tap (flipped).
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include "sac_ctx.h"
#include "speed.cuh"

using namespace sac;

namespace {

constexpr int NLAYER = 4;
constexpr int CIN_REAL[NLAYER] = {8, 32, 32, 32};
constexpr int COUT_REAL[NLAYER] = {32, 32, 32, 6};
constexpr int CIN_PAD[NLAYER] = {16, 32, 32, 32};
constexpr int COUT_PAD[NLAYER] = {32, 32, 32, 8};
constexpr int TH = 8, TW = 16;               // pixel tile: 8 rows x 16 columns
constexpr int HH = TH + 2, HW = TW + 2;      // halo tile
constexpr int NTHR = 128;

long long param_offset(int layer)            // flat FP32 order: W[cout][cin][3][3], then b[cout], per layer
{
    long long o = 0;
    for (int k = 0; k < layer; ++k) o += (long long)COUT_REAL[k] * CIN_REAL[k] * 9 + COUT_REAL[k];
    return o;
}
constexpr long long kParams = 32 * 8 * 9 + 32 + 2 * (32 * 32 * 9 + 32) + 6 * 32 * 9 + 6;   // 22566

// ---- ldmatrix / mma helpers (inline PTX) ---------------------------------------
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void ldsm_x4(unsigned addr, unsigned& r0, unsigned& r1, unsigned& r2, unsigned& r3)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3) : "r"(addr));
}
__device__ __forceinline__ void ldsm_x4_t(unsigned addr, unsigned& r0, unsigned& r1, unsigned& r2, unsigned& r3)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3) : "r"(addr));
}
__device__ __forceinline__ void ldsm_x2(unsigned addr, unsigned& r0, unsigned& r1)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];" : "=r"(r0), "=r"(r1) : "r"(addr));
}
__device__ __forceinline__ void ldsm_x2_t(unsigned addr, unsigned& r0, unsigned& r1)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];" : "=r"(r0), "=r"(r1) : "r"(addr));
}
__device__ __forceinline__ void mma_bf16(float (&d)[4], unsigned a0, unsigned a1, unsigned a2, unsigned a3,
                                         unsigned b0, unsigned b1)
{
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}
__device__ __forceinline__ void cp16(void* s, const void* g)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" :: "r"(smem_u32(s)), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;" ::: "memory"); }

// XOR swizzle of the 16-byte chunks of one pixel row: 8 consecutive rows of an
// ldmatrix land in 8 different bank groups for 2 or 4 chunks per row.
template <int CPP>
__device__ __forceinline__ int swz(int row, int chunk) { return row * CPP + (chunk ^ ((row / (8 / CPP)) % CPP)); }

__device__ __forceinline__ int wrapm(int i, int n) { int r = i % n; return r < 0 ? r + n : r; }

// Load the (TH+2) x (TW+2) periodic halo tile of an NHWC bf16 image with C
// channels into shared memory (swizzled 16-byte chunks).
template <int C>
__device__ __forceinline__ void load_halo(const __nv_bfloat16* __restrict__ img, int H, int W, int y0, int x0,
                                          __nv_bfloat16* tile)
{
    constexpr int CPP = C / 8;
    for (int v = threadIdx.x; v < HH * HW * CPP; v += NTHR) {
        const int p = v / CPP, ch = v - p * CPP;
        const int ty = p / HW, tx = p - ty * HW;
        const int gy = wrapm(y0 - 1 + ty, H), gx = wrapm(x0 - 1 + tx, W);
        cp16(tile + swz<CPP>(p, ch) * 8, img + ((long long)gy * W + gx) * C + ch * 8);
    }
}

// ---- implicit-GEMM periodic 3x3 convolution ------------------------------------
enum { MODE_RELU = 0, MODE_LINEAR_F32 = 1, MODE_MASK = 2 };

struct ConvArgs {
    const __nv_bfloat16* in;    // [H*W][CIN]
    const __nv_bfloat16* w;     // [COUT][9][CIN]
    const float* bias;          // [COUT] or null
    void* out;                  // bf16 [H*W][COUT] (RELU, MASK) or float [H*W][COUT] (LINEAR_F32)
    const __nv_bfloat16* mask;  // MASK: [H*W][COUT], output kept where mask > 0
    int H, W;
};

template <int CIN, int COUT, int MODE>
__global__ void __launch_bounds__(NTHR) conv3x3_kernel(const ConvArgs a)
{
    constexpr int CPP = CIN / 8;                 // 16-byte chunks per pixel
    constexpr int WROW = 9 * CIN + 8;            // weight row (elements), padded to an odd number of chunks
    constexpr int NT = COUT / 8;                 // n-tiles
    extern __shared__ __align__(16) unsigned char smem[];
    __nv_bfloat16* sw = reinterpret_cast<__nv_bfloat16*>(smem);                 // [COUT][WROW]
    __nv_bfloat16* st = sw + COUT * WROW;                                       // [HH*HW][CIN] swizzled
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    for (int v = threadIdx.x; v < COUT * 9 * CPP; v += NTHR) {
        const int o = v / (9 * CPP), ch = v - o * 9 * CPP;
        cp16(sw + o * WROW + ch * 8, a.w + (long long)o * 9 * CIN + ch * 8);
    }
    const int tiles_x = (a.W + TW - 1) / TW, tiles_y = (a.H + TH - 1) / TH;
    for (int tile = blockIdx.x; tile < tiles_x * tiles_y; tile += gridDim.x) {
        const int y0 = (tile / tiles_x) * TH, x0 = (tile % tiles_x) * TW;
        __syncthreads();                               // previous tile's readers are done
        load_halo<CIN>(a.in, a.H, a.W, y0, x0, st);
        cp_wait();
        __syncthreads();
        float acc[2][NT][4];
#pragma unroll
        for (int m = 0; m < 2; ++m)
#pragma unroll
            for (int n = 0; n < NT; ++n)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[m][n][q] = 0.f;
#pragma unroll
        for (int tap = 0; tap < 9; ++tap) {
            const int dy = tap / 3, dx = tap % 3;
#pragma unroll
            for (int kk = 0; kk < CIN / 16; ++kk) {
                unsigned af[2][4];
#pragma unroll
                for (int m = 0; m < 2; ++m) {
                    const int py = warp * 2 + m;
                    const int p = (py + dy) * HW + dx + (lane & 15);
                    ldsm_x4(smem_u32(st + swz<CPP>(p, kk * 2 + (lane >> 4)) * 8), af[m][0], af[m][1], af[m][2], af[m][3]);
                }
#pragma unroll
                for (int n = 0; n < NT; ++n) {
                    unsigned b0, b1;
                    const int o = n * 8 + (lane & 7);
                    ldsm_x2(smem_u32(sw + o * WROW + tap * CIN + kk * 16 + ((lane >> 3) & 1) * 8), b0, b1);
#pragma unroll
                    for (int m = 0; m < 2; ++m) mma_bf16(acc[m][n], af[m][0], af[m][1], af[m][2], af[m][3], b0, b1);
                }
            }
        }
        // epilogue: C fragment rows = pixels g and g+8 of the m-tile, cols = 2 channels
        const int g = lane >> 2, t2 = (lane & 3) * 2;
#pragma unroll
        for (int m = 0; m < 2; ++m) {
            const int gy = y0 + warp * 2 + m;
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                const int gx = x0 + g + half * 8;
                if (gy >= a.H || gx >= a.W) continue;
                const long long pix = (long long)gy * a.W + gx;
#pragma unroll
                for (int n = 0; n < NT; ++n) {
                    const int o = n * 8 + t2;
                    float v0 = acc[m][n][half * 2 + 0], v1 = acc[m][n][half * 2 + 1];
                    if (MODE != MODE_MASK && a.bias) { v0 += a.bias[o]; v1 += a.bias[o + 1]; }
                    if (MODE == MODE_RELU) { v0 = fmaxf(v0, 0.f); v1 = fmaxf(v1, 0.f); }
                    if (MODE == MODE_MASK) {
                        const __nv_bfloat162 mk = *reinterpret_cast<const __nv_bfloat162*>(a.mask + pix * COUT + o);
                        if (!(__bfloat162float(mk.x) > 0.f)) v0 = 0.f;
                        if (!(__bfloat162float(mk.y) > 0.f)) v1 = 0.f;
                    }
                    if (MODE == MODE_LINEAR_F32) {
                        *reinterpret_cast<float2*>(reinterpret_cast<float*>(a.out) + pix * COUT + o) = make_float2(v0, v1);
                    } else {
                        *reinterpret_cast<__nv_bfloat162*>(reinterpret_cast<__nv_bfloat16*>(a.out) + pix * COUT + o) =
                            __floats2bfloat162_rn(v0, v1);
                    }
                }
            }
        }
    }
}

// ---- tcgen05 implicit-GEMM periodic 3x3 convolution ------------------------------
// The same convolution on the 5th-generation tensor cores.  One CTA of 128
// threads owns a tile of TP = 128 consecutive pixels of one image row: the GEMM
// has M = 128 (pixels), N = NC (output channels, COUT padded to 16 or 32) and
// K = 9 taps x CIN channels.  Per tap and 16-channel step one
// tcgen05.mma.cta_group::1.kind::f16 (BF16 operands in shared memory, FP32
// accumulator of 128 lanes x NC columns in tensor memory) is issued by one
// thread; the epilogue reads the accumulator back with tcgen05.ld (warp w owns
// lanes 32w .. 32w+31, i.e. pixels 32w .. 32w+31 of the tile).
// Shared-memory operands use the K-major layout without swizzle, in 8-row x
// 16-byte core matrices:
//   halo  [3 rows][CIN/8 chunks][HP pixels][8 ch]: the A operand of tap (dy, dx)
//         starts at row dy, pixel dx; consecutive pixels are 16 B apart, so 8
//         pixels form one core matrix (SBO = 128 B between pixel groups) and the
//         next 8 channels are HP * 16 B away (LBO);
//   wts   [9 taps][CIN/8 chunks][NC/8 groups][8 out ch][8 ch]: the B operand
//         (SBO = 128 B between output-channel groups, LBO = NC/8 * 128 B).
namespace tcv {
constexpr int TP = 128, HP = TP + 2, NTHR_TC = 128;

__device__ __forceinline__ unsigned long long smem_desc(unsigned addr, unsigned lbo, unsigned sbo)
{
    // start address, leading / stride byte offsets (16-byte units), descriptor
    // version 1 (bits 46-47), no swizzle, base offset 0
    return (unsigned long long)((addr & 0x3FFFFu) >> 4) | ((unsigned long long)((lbo >> 4) & 0x3FFFu) << 16) |
           ((unsigned long long)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
// instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N = n, M = 128
__host__ __device__ constexpr unsigned idesc_bf16(int n)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(n >> 3) << 17) | ((unsigned)(128 >> 4) << 24);
}
__device__ __forceinline__ void mma_bf16_tc(unsigned tmem_d, unsigned long long adesc, unsigned long long bdesc,
                                            unsigned idesc, int accumulate)
{
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                 " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
                 :: "r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate) : "memory");
}
__device__ __forceinline__ void mbar_init_tc(unsigned long long* bar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ bool mbar_wait_tc(unsigned long long* bar, unsigned parity)
{
    unsigned long long t0 = 0;
    for (;;) {
        // the clock is read once per 32 polls: polling is what finds the phase complete
        for (int k = 0; k < 32; ++k) {
            unsigned ok;
            asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                         : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
            if (ok) return true;
        }
        unsigned long long t;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        if (t0 == 0) t0 = t;
        else if (t - t0 > 1000000000ull) return false;   // about one second
    }
}

constexpr int ROWS = 4;   // image rows per tile: four independent 128 x NC accumulators

template <int CIN, int NC>
struct TcSmem {
    static constexpr int CPP = CIN / 8, NG = NC / 8;
    static constexpr int HALO_BYTES = (ROWS + 2) * CPP * HP * 16;
    static constexpr int W_BYTES = 9 * CPP * NG * 128;
    static constexpr int BYTES = HALO_BYTES + W_BYTES + 64;   // + mbarrier, TMEM address
    static constexpr int TMEM_COLS = ROWS * NC <= 32 ? 32 : (ROWS * NC <= 64 ? 64 : 128);
};

// Copy the halo of a tile (rows y0-1 .. y0+ROWS, pixels x0-1 .. x0+TP, periodic)
// with 16-byte cp.async.
template <int CIN>
__device__ __forceinline__ void stage_halo_tc(const ConvArgs& a, int y0, int x0, unsigned char* halo)
{
    constexpr int CPP = CIN / 8;
#pragma unroll
    for (int r = 0; r < ROWS + 2; ++r) {
        int gy = y0 - 1 + r;
        gy = gy < 0 ? gy + a.H : (gy >= a.H ? gy - a.H : gy);
        const __nv_bfloat16* row = a.in + (long long)gy * a.W * CIN;
        for (int v = threadIdx.x; v < CPP * HP; v += NTHR_TC) {
            const int ch = v / HP, px = v - ch * HP;
            int gx = x0 - 1 + px;
            gx = gx < 0 ? gx + a.W : (gx >= a.W ? gx - a.W : gx);
            cp16(halo + ((r * CPP + ch) * HP + px) * 16, row + (long long)gx * CIN + ch * 8);
        }
    }
}

// Epilogue of one accumulator row: tensor-memory columns q*NC .. q*NC+NC-1 of
// this warp's 32 lanes (pixels), bias / ReLU / mask, stored as NHWC (BF16 or
// FP32); image row gy, this thread's pixel gx (nothing is stored outside the
// image).  sb: the layer's bias staged in shared memory (read when a.bias is set).
template <int COUT, int NC, int MODE>
__device__ __forceinline__ void epilogue_row(const ConvArgs& a, const float* __restrict__ sb, unsigned tmem, int warp,
                                             int q, int gy, int gx)
{
    float acc[NC];
    {
        unsigned r[NC];
        const unsigned taddr = tmem + ((unsigned)(warp * 32) << 16) + q * NC;
        if constexpr (NC == 32) {
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                         "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                         "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                         : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                           "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
                           "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
                           "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
                           "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
                           "=r"(r[31])
                         : "r"(taddr) : "memory");
        } else {
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                         "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                         : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                           "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
                           "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                         : "r"(taddr) : "memory");
        }
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int o = 0; o < NC; ++o) acc[o] = __uint_as_float(r[o]);
    }
    if (gx >= a.W || gy >= a.H) return;
    const long long pix = (long long)gy * a.W + gx;
    if (MODE == MODE_LINEAR_F32) {
        float* out = reinterpret_cast<float*>(a.out) + pix * COUT;
#pragma unroll
        for (int o = 0; o < COUT; o += 4)
            *reinterpret_cast<float4*>(out + o) =
                make_float4(acc[o] + sb[o], acc[o + 1] + sb[o + 1], acc[o + 2] + sb[o + 2], acc[o + 3] + sb[o + 3]);
    } else {
        __align__(16) __nv_bfloat162 ov[COUT / 2];
#pragma unroll
        for (int o = 0; o < COUT; o += 2) {
            float v0 = acc[o], v1 = acc[o + 1];
            if (MODE == MODE_RELU) {
                if (a.bias) { v0 += sb[o]; v1 += sb[o + 1]; }
                v0 = fmaxf(v0, 0.f); v1 = fmaxf(v1, 0.f);
            } else {   // MODE_MASK: keep where the layer's activation is positive
                const __nv_bfloat162 mk = *reinterpret_cast<const __nv_bfloat162*>(a.mask + pix * COUT + o);
                if (!(__bfloat162float(mk.x) > 0.f)) v0 = 0.f;
                if (!(__bfloat162float(mk.y) > 0.f)) v1 = 0.f;
            }
            ov[o / 2] = __floats2bfloat162_rn(v0, v1);
        }
        uint4* dst = reinterpret_cast<uint4*>(reinterpret_cast<__nv_bfloat16*>(a.out) + pix * COUT);
#pragma unroll
        for (int k = 0; k < COUT / 8; ++k) dst[k] = reinterpret_cast<const uint4*>(ov)[k];
    }
}

// COUT: channels stored (<= NC); the weight rows COUT .. NC-1 are zero.  A tile
// is ROWS image rows x TP pixels: row q accumulates into tensor-memory columns
// q*NC .. q*NC+NC-1, and its MMAs are issued interleaved with the other rows'
// (independent accumulators keep the tensor pipe busy).  Rows past the image
// (the last tile of a height that ROWS does not divide) are computed on wrapped
// rows and not stored.
template <int CIN, int COUT, int NC, int MODE>
__global__ void __launch_bounds__(NTHR_TC) conv3x3_tc_kernel(const ConvArgs a, int* err)
{
    using L = TcSmem<CIN, NC>;
    constexpr int CPP = L::CPP, NG = L::NG;
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char* halo = smem;
    unsigned char* wts = smem + L::HALO_BYTES;
    unsigned long long* bar = reinterpret_cast<unsigned long long*>(smem + L::HALO_BYTES + L::W_BYTES);
    unsigned* tmem_slot = reinterpret_cast<unsigned*>(smem + L::HALO_BYTES + L::W_BYTES + 8);
    const int tid = threadIdx.x, warp = tid >> 5;

    // weights: 16-byte chunks (o, tap, chunk) of the [COUT][9][CIN] layout
    for (int v = tid; v < NC * 9 * CPP; v += NTHR_TC) {
        const int o = v / (9 * CPP), rem = v - o * 9 * CPP, tap = rem / CPP, ch = rem - tap * CPP;
        unsigned char* dst = wts + ((tap * CPP + ch) * NG + (o >> 3)) * 128 + (o & 7) * 16;
        if (o < COUT) cp16(dst, a.w + ((long long)o * 9 + tap) * CIN + ch * 8);
        else *reinterpret_cast<uint4*>(dst) = make_uint4(0, 0, 0, 0);
    }
    __shared__ float s_bias[NC];
    if (tid < NC) s_bias[tid] = (a.bias && tid < COUT) ? a.bias[tid] : 0.f;   // visible after the barrier below
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(tmem_slot)), "r"(L::TMEM_COLS) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) mbar_init_tc(bar);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned tmem = *tmem_slot;
    const unsigned wbase = smem_u32(wts), hbase = smem_u32(halo);
    constexpr unsigned IDESC = idesc_bf16(NC);

    const int tiles_x = (a.W + TP - 1) / TP, tiles_y = (a.H + ROWS - 1) / ROWS, ntiles = tiles_x * tiles_y;
    unsigned phase = 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int ty = tile / tiles_x, x0 = (tile - ty * tiles_x) * TP, y0 = ty * ROWS;
        stage_halo_tc<CIN>(a, y0, x0, halo);
        cp_wait();
        // make the generic-proxy writes visible to the tensor core (async proxy)
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int tap = 0; tap < 9; ++tap) {
                const int dy = tap / 3, dx = tap - dy * 3;
#pragma unroll
                for (int ks = 0; ks < CPP / 2; ++ks) {
                    const unsigned baddr = wbase + ((tap * CPP + 2 * ks) * NG) * 128;
                    const unsigned long long bdesc = smem_desc(baddr, NG * 128, 128);
#pragma unroll
                    for (int q = 0; q < ROWS; ++q) {
                        const unsigned aaddr = hbase + (((q + dy) * CPP + 2 * ks) * HP + dx) * 16;
                        mma_bf16_tc(tmem + q * NC, smem_desc(aaddr, HP * 16, 128), bdesc, IDESC, (tap | ks) != 0);
                    }
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         :: "r"(smem_u32(bar)) : "memory");
        }
        __syncwarp();
        const bool done = mbar_wait_tc(bar, phase);
        phase ^= 1u;
        if (__syncthreads_or(!done)) {   // the accumulators never arrived: report, do not read them
            if (tid == 0) atomicExch(err, 1);
            break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int gx = x0 + tid;
#pragma unroll 1
        for (int q = 0; q < ROWS; ++q) epilogue_row<COUT, NC, MODE>(a, s_bias, tmem, warp, q, y0 + q, gx);
        // the accumulators and the halo are reused by the next tile once every warp is done
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(L::TMEM_COLS) : "memory");
}
// The same convolution fed by tensor-map copies and software-pipelined: a tile
// is RT image rows x TP pixels; each of its RT+2 halo rows arrives by one 4D
// tensor copy ((8 channels, pixel, 8-channel chunk, row) of the NHWC image, so
// the copy lands in the [chunk][pixel][8 ch] core-matrix layout directly) into
// one of two halo buffers, and the tile's MMAs accumulate into one of two
// tensor-memory accumulators.  While the MMAs of tile i run, the threads write
// back tile i-1 and the copies of tile i+1 are in flight.  Pixels left of
// column 0 or right of column W-1 read zeros and are then patched with the
// periodic neighbour column.
template <int CIN, int NC, int RT>
struct TmaSmem {
    static constexpr int CPP = CIN / 8, NG = NC / 8;
    static constexpr int ROW_BYTES = CPP * HP * 16;                    // one row's copy (dense)
    static constexpr int ROW_STRIDE = (ROW_BYTES + 127) / 128 * 128;   // row copies start 128-byte aligned
    static constexpr int HALO_BYTES = (RT + 2) * ROW_STRIDE;
    static constexpr int W_BYTES = 9 * CPP * NG * 128;
    static constexpr int BYTES = 128 + 2 * HALO_BYTES + W_BYTES + 64;   // + alignment of the base
    static constexpr int ACC_COLS = RT * NC;                           // one accumulator
    static constexpr int TMEM_COLS = 2 * ACC_COLS <= 32 ? 32 : (2 * ACC_COLS <= 64 ? 64 : 128);
};

__device__ __forceinline__ void mbar_expect_tc(unsigned long long* bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// One thread: the RT+2 row copies of the tile whose top-left output pixel is
// (x0, y0) into a halo buffer; completion on bar.
template <int CIN, int NC, int RT>
__device__ __forceinline__ void issue_halo_tma(const CUtensorMap* tm, const ConvArgs& a, int y0, int x0,
                                               unsigned char* halo, unsigned long long* bar)
{
    using L = TmaSmem<CIN, NC, RT>;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect_tc(bar, (unsigned)((RT + 2) * L::ROW_BYTES));
#pragma unroll
    for (int r = 0; r < RT + 2; ++r) {
        int gy = y0 - 1 + r;
        gy = gy < 0 ? gy + a.H : (gy >= a.H ? gy - a.H : gy);
        asm volatile("cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes"
                     " [%0], [%1, {%2, %3, %4, %5}], [%6];"
                     :: "r"(smem_u32(halo + r * L::ROW_STRIDE)), "l"(tm), "r"(0), "r"(x0 - 1), "r"(0), "r"(gy),
                        "r"(smem_u32(bar)) : "memory");
    }
}

template <int CIN, int COUT, int NC, int MODE, int RT>
__global__ void __launch_bounds__(NTHR_TC) conv3x3_tma_kernel(const ConvArgs a, const __grid_constant__ CUtensorMap tm,
                                                              int* err)
{
    using L = TmaSmem<CIN, NC, RT>;
    constexpr int CPP = L::CPP, NG = L::NG;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char* smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);   // 128-byte aligned base
    unsigned char* wts = smem + 2 * L::HALO_BYTES;
    unsigned long long* bar = reinterpret_cast<unsigned long long*>(smem + 2 * L::HALO_BYTES + L::W_BYTES);
    // bar[0], bar[1]: halo buffer landed; bar[2], bar[3]: accumulator complete
    unsigned* tmem_slot = reinterpret_cast<unsigned*>(smem + 2 * L::HALO_BYTES + L::W_BYTES + 32);
    const int tid = threadIdx.x, warp = tid >> 5;

    for (int v = tid; v < NC * 9 * CPP; v += NTHR_TC) {
        const int o = v / (9 * CPP), rem = v - o * 9 * CPP, tap = rem / CPP, ch = rem - tap * CPP;
        unsigned char* dst = wts + ((tap * CPP + ch) * NG + (o >> 3)) * 128 + (o & 7) * 16;
        if (o < COUT) cp16(dst, a.w + ((long long)o * 9 + tap) * CIN + ch * 8);
        else *reinterpret_cast<uint4*>(dst) = make_uint4(0, 0, 0, 0);
    }
    cp_wait();
    __shared__ float s_bias[NC];
    if (tid < NC) s_bias[tid] = (a.bias && tid < COUT) ? a.bias[tid] : 0.f;   // visible after the barrier below
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(tmem_slot)), "r"(L::TMEM_COLS) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0)
        for (int k = 0; k < 4; ++k) mbar_init_tc(&bar[k]);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // the weights, for the tensor core
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned tmem = *tmem_slot;
    const unsigned wbase = smem_u32(wts);
    constexpr unsigned IDESC = idesc_bf16(NC);

    const int tiles_x = (a.W + TP - 1) / TP, tiles_y = (a.H + RT - 1) / RT, ntiles = tiles_x * tiles_y;
    const int first = blockIdx.x, n = first < ntiles ? (ntiles - 1 - first) / (int)gridDim.x + 1 : 0;
    auto tile_of = [&](int i) { return first + i * (int)gridDim.x; };
    // per buffer / accumulator k (bit k): phase of the next wait on its copies
    // (lph) and on its MMAs (mph), copies in flight (infl), MMAs not yet waited (pend)
    unsigned lph = 0u, mph = 0u, infl = 0u, pend = 0u;
    auto halo = [&](int k) { return smem + k * L::HALO_BYTES; };
    if (n > 0) {
        if (tid == 0) issue_halo_tma<CIN, NC, RT>(&tm, a, (first / tiles_x) * RT, (first % tiles_x) * TP, halo(0), &bar[0]);
        infl |= 1u;
    }
    bool ok = true;
    for (int i = 0; i <= n && ok; ++i) {
        const int b = i & 1;
        if (i < n) {
            // ---- tile i: copies landed, periodic columns, MMAs into accumulator b
            const int t = tile_of(i), y0 = (t / tiles_x) * RT, x0 = (t % tiles_x) * TP;
            const bool landed = mbar_wait_tc(&bar[b], (lph >> b) & 1u);
            if (landed) { lph ^= 1u << b; infl &= ~(1u << b); }
            if (__syncthreads_or(!landed)) { ok = false; break; }
            const int pr = a.W - x0 + 1;
            for (int v = tid; v < 2 * (RT + 2) * CPP; v += NTHR_TC) {
                const int side = v / ((RT + 2) * CPP), rem = v - side * (RT + 2) * CPP, r = rem / CPP, ch = rem - r * CPP;
                if ((side == 0 && x0 != 0) || (side == 1 && pr > HP - 1)) continue;
                int gy = y0 - 1 + r;
                gy = gy < 0 ? gy + a.H : (gy >= a.H ? gy - a.H : gy);
                const int px = side == 0 ? 0 : pr, gx = side == 0 ? a.W - 1 : 0;
                *reinterpret_cast<uint4*>(halo(b) + r * L::ROW_STRIDE + (ch * HP + px) * 16) =
                    *reinterpret_cast<const uint4*>(a.in + ((long long)gy * a.W + gx) * CIN + ch * 8);
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncthreads();
            if (tid == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const unsigned hbase = smem_u32(halo(b)), acc = tmem + b * L::ACC_COLS;
#pragma unroll
                for (int tap = 0; tap < 9; ++tap) {
                    const int dy = tap / 3, dx = tap - dy * 3;
#pragma unroll
                    for (int ks = 0; ks < CPP / 2; ++ks) {
                        const unsigned long long bdesc = smem_desc(wbase + ((tap * CPP + 2 * ks) * NG) * 128, NG * 128, 128);
#pragma unroll
                        for (int q = 0; q < RT; ++q) {
                            const unsigned aaddr = hbase + (q + dy) * L::ROW_STRIDE + ((2 * ks) * HP + dx) * 16;
                            mma_bf16_tc(acc + q * NC, smem_desc(aaddr, HP * 16, 128), bdesc, IDESC, (tap | ks) != 0);
                        }
                    }
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                             :: "r"(smem_u32(&bar[2 + b])) : "memory");
            }
            pend |= 1u << b;
        }
        if (i >= 1) {
            // ---- tile i-1: its MMAs are done, so its halo buffer takes tile i+1's
            // copies; then its accumulator is written back
            const int pb = b ^ 1, t = tile_of(i - 1), y0 = (t / tiles_x) * RT, x0 = (t % tiles_x) * TP;
            __syncwarp();
            const bool done = mbar_wait_tc(&bar[2 + pb], (mph >> pb) & 1u);
            if (done) { mph ^= 1u << pb; pend &= ~(1u << pb); }
            if (__syncthreads_or(!done)) { ok = false; break; }
            if (i + 1 < n) {
                const int nt = tile_of(i + 1);
                if (tid == 0)
                    issue_halo_tma<CIN, NC, RT>(&tm, a, (nt / tiles_x) * RT, (nt % tiles_x) * TP, halo(pb), &bar[pb]);
                infl |= 1u << pb;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll 1
            for (int q = 0; q < RT; ++q)
                epilogue_row<COUT, NC, MODE>(a, s_bias, tmem + pb * L::ACC_COLS, warp, q, y0 + q, x0 + tid);
            // accumulator pb is reused by tile i+1 once every warp has read it
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncthreads();
        } else if (n > 1) {
            // tile 1's copies go to the second halo buffer, unused so far
            if (tid == 0) {
                const int nt = tile_of(1);
                issue_halo_tma<CIN, NC, RT>(&tm, a, (nt / tiles_x) * RT, (nt % tiles_x) * TP, halo(1), &bar[1]);
            }
            infl |= 2u;
        }
    }
    if (!ok && tid == 0) atomicExch(err, 1);
    // nothing may land in shared or tensor memory after the CTA has left: wait
    // (bounded) for copies and MMAs still in flight
    for (int k = 0; k < 2; ++k) {
        if ((infl >> k) & 1u) mbar_wait_tc(&bar[k], (lph >> k) & 1u);
        if ((pend >> k) & 1u) mbar_wait_tc(&bar[2 + k], (mph >> k) & 1u);
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(L::TMEM_COLS) : "memory");
}

}  // namespace tcv

// ---- weight gradient: dW[o][tap][c] = sum_p dY[p][o] X[p + tap][c] ---------------
struct DwArgs {
    const __nv_bfloat16* dy;   // [H*W][MO]
    const __nv_bfloat16* x;    // [H*W][CIN]
    float* part;               // [gridDim.x][MO][9*CIN]
    float* dbpart;             // [gridDim.x][MO]
    int H, W;
};

template <int CIN, int MO>
__global__ void __launch_bounds__(NTHR) conv3x3_dw_kernel(const DwArgs a)
{
    constexpr int CPPX = CIN / 8, CPPY = MO / 8;
    constexpr int NTOT = 9 * CIN / 8;                  // n-tiles of 8 over (tap, c)
    constexpr int NPW = (NTOT + 3) / 4;                // n-tiles per warp
    constexpr int MT = MO / 16;                        // m-tiles of 16 over o
    extern __shared__ __align__(16) unsigned char smem[];
    __nv_bfloat16* sx = reinterpret_cast<__nv_bfloat16*>(smem);                 // halo tile [HH*HW][CIN]
    __nv_bfloat16* sd = sx + HH * HW * CIN;                                     // dY tile [TH*TW][MO]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float acc[MT][NPW][4];
#pragma unroll
    for (int m = 0; m < MT; ++m)
#pragma unroll
        for (int n = 0; n < NPW; ++n)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[m][n][q] = 0.f;
    float db = 0.f;

    const int tiles_x = (a.W + TW - 1) / TW, tiles_y = (a.H + TH - 1) / TH;
    for (int tile = blockIdx.x; tile < tiles_x * tiles_y; tile += gridDim.x) {
        const int y0 = (tile / tiles_x) * TH, x0 = (tile % tiles_x) * TW;
        __syncthreads();
        load_halo<CIN>(a.x, a.H, a.W, y0, x0, sx);
        for (int v = threadIdx.x; v < TH * TW * CPPY; v += NTHR) {
            const int p = v / CPPY, ch = v - p * CPPY;
            const int gy = y0 + p / TW, gx = x0 + p % TW;
            __nv_bfloat16* dst = sd + swz<CPPY>(p, ch) * 8;
            if (gy < a.H && gx < a.W) cp16(dst, a.dy + ((long long)gy * a.W + gx) * MO + ch * 8);
            else *reinterpret_cast<uint4*>(dst) = make_uint4(0, 0, 0, 0);   // pixels outside the image add nothing
        }
        cp_wait();
        __syncthreads();
        if (threadIdx.x < MO) {
            const int o = threadIdx.x;
            for (int p = 0; p < TH * TW; ++p)
                db += __bfloat162float(sd[swz<CPPY>(p, o >> 3) * 8 + (o & 7)]);
        }
#pragma unroll
        for (int ks = 0; ks < TH; ++ks) {              // k-step: the 16 pixels of tile row ks
            unsigned af[MT][4];
#pragma unroll
            for (int m = 0; m < MT; ++m) {
                // A[o][p] = dY[p][o]: stored rows p, transposed load; matrix j = lane>>3
                const int j = lane >> 3;
                const int p = ks * TW + (j >> 1) * 8 + (lane & 7);
                const int ch = m * 2 + (j & 1);
                ldsm_x4_t(smem_u32(sd + swz<CPPY>(p, ch) * 8), af[m][0], af[m][1], af[m][2], af[m][3]);
            }
#pragma unroll
            for (int nn = 0; nn < NPW; ++nn) {
                const int nt = warp + nn * 4;
                if (nt >= NTOT) break;
                const int tap = (nt * 8) / CIN, c0 = (nt * 8) % CIN;
                const int dyy = tap / 3, dxx = tap % 3;
                // B[p][(tap,c)] = X[p + tap][c]: stored rows p (halo pixels), transposed load
                const int hp = (ks + dyy) * HW + dxx + ((lane >> 3) & 1) * 8 + (lane & 7);
                unsigned b0, b1;
                ldsm_x2_t(smem_u32(sx + swz<CPPX>(hp, c0 / 8) * 8), b0, b1);
#pragma unroll
                for (int m = 0; m < MT; ++m) mma_bf16(acc[m][nn], af[m][0], af[m][1], af[m][2], af[m][3], b0, b1);
            }
        }
    }
    // partials of this CTA: C rows = o (g, g+8), cols = n (2 per lane)
    const int g = lane >> 2, t2 = (lane & 3) * 2;
    float* out = a.part + (long long)blockIdx.x * MO * 9 * CIN;
#pragma unroll
    for (int m = 0; m < MT; ++m)
#pragma unroll
        for (int nn = 0; nn < NPW; ++nn) {
            const int nt = warp + nn * 4;
            if (nt >= NTOT) break;
            const int n = nt * 8 + t2;
            out[(m * 16 + g) * 9 * CIN + n] = acc[m][nn][0];
            out[(m * 16 + g) * 9 * CIN + n + 1] = acc[m][nn][1];
            out[(m * 16 + g + 8) * 9 * CIN + n] = acc[m][nn][2];
            out[(m * 16 + g + 8) * 9 * CIN + n + 1] = acc[m][nn][3];
        }
    if (threadIdx.x < MO) a.dbpart[(long long)blockIdx.x * MO + threadIdx.x] = db;
}

// Sum the per-CTA partials in a fixed order into the flat FP32 gradient of one layer.
__global__ void dw_reduce_kernel(const float* __restrict__ part, const float* __restrict__ dbpart, int nblk,
                                 int cin_pad, int mo_pad, int cin, int cout, float* __restrict__ gw,
                                 float* __restrict__ gb)
{
    const int nw = cout * cin * 9;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < nw + cout; v += gridDim.x * blockDim.x) {
        float s = 0.f;
        if (v < nw) {
            const int o = v / (cin * 9), rem = v - o * cin * 9, c = rem / 9, tap = rem % 9;
            const long long idx = (long long)o * 9 * cin_pad + tap * cin_pad + c;
            for (int b = 0; b < nblk; ++b) s += part[(long long)b * mo_pad * 9 * cin_pad + idx];
            gw[v] = s;
        } else {
            const int o = v - nw;
            for (int b = 0; b < nblk; ++b) s += dbpart[(long long)b * mo_pad + o];
            gb[o] = s;
        }
    }
}

// FP32 master parameters -> bf16 forward weights [COUTP][9][CINP] and flipped,
// transposed input-gradient weights [CINP][9][COUTP] (padding zero), FP32 bias.
__global__ void pack_weights_kernel(const float* __restrict__ params, int cin, int cout, int cinp, int coutp,
                                    int coutp_t, __nv_bfloat16* __restrict__ wf, __nv_bfloat16* __restrict__ wt,
                                    float* __restrict__ bias)
{
    const int n = coutp * 9 * cinp;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const int o = v / (9 * cinp), rem = v - o * 9 * cinp, tap = rem / cinp, c = rem % cinp;
        const float w = (o < cout && c < cin) ? params[(o * cin + c) * 9 + tap] : 0.f;
        const __nv_bfloat16 wb = __float2bfloat16_rn(w);
        wf[v] = wb;
        if (wt) wt[((long long)c * 9 + (8 - tap)) * coutp_t + o] = wb;   // padding rows o >= coutp stay zero
    }
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < coutp; v += gridDim.x * blockDim.x)
        bias[v] = v < cout ? params[(long long)cout * cin * 9 + v] : 0.f;
}

// 8 input features (normalised) from a packed FP32 conserved state [6][H][W],
// periodic: rho, m_x, m_y, e, B_x, B_y, p_k, j_z = D_x B_y - D_y B_x (section 2
// fourth-order differences); channels 8..15 are zero padding.
__global__ void features_kernel(const float* __restrict__ w, int H, int W, float gm1, float inv12dx, float inv12dy,
                                const float* __restrict__ scale, __nv_bfloat16* __restrict__ out)
{
    const long long n = (long long)H * W;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(p / W), i = (int)(p % W);
        const float rho = w[p], mx = w[n + p], my = w[2 * n + p], e = w[3 * n + p], bx = w[4 * n + p], by = w[5 * n + p];
        const float pk = gm1 * (e - 0.5f * (mx * mx + my * my) / rho - 0.5f * (bx * bx + by * by));
        const float* BY = w + 5 * n + (long long)j * W;
        const float dby = (8.f * (BY[wrapm(i + 1, W)] - BY[wrapm(i - 1, W)]) - (BY[wrapm(i + 2, W)] - BY[wrapm(i - 2, W)])) * inv12dx;
        const float* BX = w + 4 * n + i;
        const float dbx = (8.f * (BX[(long long)wrapm(j + 1, H) * W] - BX[(long long)wrapm(j - 1, H) * W]) -
                           (BX[(long long)wrapm(j + 2, H) * W] - BX[(long long)wrapm(j - 2, H) * W])) * inv12dy;
        const float f[8] = {rho, mx, my, e, bx, by, pk, dby - dbx};
        __align__(16) __nv_bfloat16 o[16];
#pragma unroll
        for (int c = 0; c < 8; ++c) o[c] = __float2bfloat16_rn(f[c] / scale[c]);
#pragma unroll
        for (int c = 8; c < 16; ++c) o[c] = __float2bfloat16_rn(0.f);
        uint4* dst = reinterpret_cast<uint4*>(out + p * 16);
        dst[0] = reinterpret_cast<const uint4*>(o)[0];
        dst[1] = reinterpret_cast<const uint4*>(o)[1];
    }
}

// Target t_c = (next_c - w_c) / out_scale_c (the residual the coarse step left);
// loss 0.5 mean (pred - t)^2 over 6 channels; dY = (pred - t) / (6 n) as bf16 [p][16]
__global__ void loss_kernel(const float* __restrict__ pred, const float* __restrict__ w,
                            const float* __restrict__ next, const float* __restrict__ out_scale, long long n,
                            __nv_bfloat16* __restrict__ dy, float* __restrict__ loss_part)
{
    __shared__ float red[NTHR / 32];
    float s = 0.f;
    const float inv = 1.f / (6.f * (float)n);
    float iscale[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) iscale[c] = 1.f / out_scale[c];
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
        __align__(16) __nv_bfloat16 o[16];
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            const float t = (next[c * n + p] - w[c * n + p]) * iscale[c];
            const float r = pred[p * 8 + c] - t;
            s += r * r;
            o[c] = __float2bfloat16_rn(r * inv);
        }
#pragma unroll
        for (int c = 6; c < 16; ++c) o[c] = __float2bfloat16_rn(0.f);
        uint4* d = reinterpret_cast<uint4*>(dy + p * 16);
        d[0] = reinterpret_cast<const uint4*>(o)[0];
        d[1] = reinterpret_cast<const uint4*>(o)[1];
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int k = 0; k < NTHR / 32; ++k) t += red[k];
        loss_part[blockIdx.x] = t;
    }
}

__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, long long n, float lr, float b1, float b2, float eps,
                            float c1, float c2)
{
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const float gk = g[k];
        const float mk = b1 * m[k] + (1.f - b1) * gk;
        const float vk = b2 * v[k] + (1.f - b2) * gk * gk;
        m[k] = mk; v[k] = vk;
        p[k] -= lr * (mk / c1) / (sqrtf(vk / c2) + eps);
    }
}

// out = w + amp_f * xi, xi ~ U[-1,1) from SplitMix64 of (seed, element index)
__global__ void perturb_kernel(const float* __restrict__ w, float* __restrict__ out, long long n_per_field,
                               const float* __restrict__ amp, unsigned long long seed)
{
    const long long total = n_per_field * NF;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < total; v += (long long)gridDim.x * blockDim.x) {
        unsigned long long z = seed + (unsigned long long)(v + 1) * 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        const float xi = 2.f * (float)((double)(z >> 11) * (1.0 / 9007199254740992.0)) - 1.f;
        out[v] = w[v] + amp[v / n_per_field] * xi;
    }
}

__global__ void block_average_kernel(const float* __restrict__ fine, int nf, int hf, int wf, int r,
                                     float* __restrict__ coarse)
{
    const int hc = hf / r, wc = wf / r;
    const long long nc = (long long)hc * wc, total = nc * nf;
    const float inv = 1.f / (float)(r * r);
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < total; v += (long long)gridDim.x * blockDim.x) {
        const int f = (int)(v / nc);
        const long long q = v - (long long)f * nc;
        const int J = (int)(q / wc), I = (int)(q % wc);
        const float* src = fine + (long long)f * hf * wf + (long long)J * r * wf + (long long)I * r;
        float s = 0.f;
        for (int a = 0; a < r; ++a)
            for (int b = 0; b < r; ++b) s += src[(long long)a * wf + b];
        coarse[v] = s * inv;
    }
}

// ---- correction of a solver context ---------------------------------------------
// fields of the three float2 planes of the FP32 layout: (rho, e), (m_x, m_y), (B_x, B_y)
__device__ __forceinline__ void plane_fields(int p, int& f0, int& f1)
{
    f0 = p == 0 ? 0 : (p == 1 ? 1 : 4);
    f1 = p == 0 ? 3 : (p == 1 ? 2 : 5);
}

// Packed [6][ny][nx] copy of the interior: one thread per (plane, cell), one
// 8-byte read of the field pair, two 4-byte writes.
__global__ void export_paired_kernel(const float* __restrict__ u0, Layout L, float* __restrict__ dst)
{
    const long long n = (long long)L.nx * L.ny;
    const float2* w = reinterpret_cast<const float2*>(u0);
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < 3 * n; v += (long long)gridDim.x * blockDim.x) {
        const int p = (int)(v / n);
        const long long r = v - (long long)p * n;
        const float2 q = w[p * L.fstride + L.at((int)(r % L.nx), (int)(r / L.nx))];
        int f0, f1;
        plane_fields(p, f0, f1);
        dst[f0 * n + r] = q.x;
        dst[f1 * n + r] = q.y;
    }
}

// The network output applied to the state, limited to [-clip, clip] (units of
// out_scale) when clip > 0.
__device__ __forceinline__ float limited(float v, float clip) { return clip > 0.f ? fminf(fmaxf(v, -clip), clip) : v; }

// Limiter of the correction of cell p (positive != 0): 1 if the corrected cell
// keeps at least half of its density and of its kinetic pressure
// p_k = (gamma-1)(e - |m|^2/(2 rho) - |B|^2/2), else 0 (no correction there).
__device__ __forceinline__ float keep_factor(const float* __restrict__ state, long long p, long long n,
                                             const float* __restrict__ pred, const float* __restrict__ osc, float clip,
                                             float gm1, int positive)
{
    if (!positive) return 1.f;
    float u[NF], v[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
        u[f] = state[f * n + p];
        v[f] = u[f] + osc[f] * limited(pred[p * 8 + f], clip);
    }
    const float pk0 = gm1 * (u[3] - 0.5f * (u[1] * u[1] + u[2] * u[2]) / u[0] - 0.5f * (u[4] * u[4] + u[5] * u[5]));
    const float pk1 = gm1 * (v[3] - 0.5f * (v[1] * v[1] + v[2] * v[2]) / v[0] - 0.5f * (v[4] * v[4] + v[5] * v[5]));
    return (v[0] > 0.5f * u[0] && pk1 > 0.5f * pk0) ? 1.f : 0.f;
}

// Per-block partial sums of the 6 (limited) output channels (fixed order; the
// final sum is taken in add_correction_kernel's prologue by every block, in the
// same order).
__global__ void pred_sum_kernel(const float* __restrict__ pred, long long n, float clip, const float* __restrict__ state,
                                const float* __restrict__ osc, float gm1, int positive, float* __restrict__ part)
{
    __shared__ float red[6][NTHR / 32];
    float s[6] = {0, 0, 0, 0, 0, 0};
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
        const float k = keep_factor(state, p, n, pred, osc, clip, gm1, positive);
#pragma unroll
        for (int c = 0; c < 6; ++c) s[c] += k * limited(pred[p * 8 + c], clip);
    }
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        float x = s[c];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if ((threadIdx.x & 31) == 0) red[c][threadIdx.x >> 5] = x;
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        float x = 0.f;
        for (int k = 0; k < NTHR / 32; ++k) x += red[threadIdx.x][k];
        part[blockIdx.x * 6 + threadIdx.x] = x;
    }
}

// u += out_scale * (p - mean(p)), p = the limited network output, on the interior
// and on every periodic ghost copy: the correction is conservative (it moves no
// mass, momentum, energy or flux in or out of the periodic domain, as the fine
// and coarse runs conserve them).
__global__ void add_correction_kernel(float* __restrict__ u0, Layout L, const float* __restrict__ pred,
                                      const float* __restrict__ out_scale, const float* __restrict__ part,
                                      int nblk, float clip, const float* __restrict__ state, float gm1, int positive,
                                      DevScalars* sc)
{
    __shared__ float mean[6];
    if (threadIdx.x < 6) {
        float x = 0.f;
        for (int b = 0; b < nblk; ++b) x += part[b * 6 + threadIdx.x];
        mean[threadIdx.x] = x / (float)((long long)L.nx * L.ny);
    }
    __syncthreads();
    if (blockIdx.x == 0 && threadIdx.x == 0) { sc->cmax_bits[0] = 0ull; sc->cmax_bits[1] = 0ull; }
    // one thread per ghost-extended cell: the limiter once, then the three field pairs
    float2* w = reinterpret_cast<float2*>(u0);
    const long long n = (long long)L.nx * L.ny;
    const long long ex = L.nx + 2 * GY, total = ex * (L.ny + 2 * GY);
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < total; v += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(v / ex) - GY, i = (int)(v % ex) - GY;
        const long long p = (long long)wrapm(j, L.ny) * L.nx + wrapm(i, L.nx);
        const float k = keep_factor(state, p, n, pred, out_scale, clip, gm1, positive);
        const long long e = L.at(i, j);
#pragma unroll
        for (int pl = 0; pl < 3; ++pl) {
            int f0, f1;
            plane_fields(pl, f0, f1);
            float2 q = w[pl * L.fstride + e];
            q.x += out_scale[f0] * (k * limited(pred[p * 8 + f0], clip) - mean[f0]);
            q.y += out_scale[f1] * (k * limited(pred[p * 8 + f1], clip) - mean[f1]);
            w[pl * L.fstride + e] = q;
        }
    }
}

__global__ void cmax_paired_kernel(const float* __restrict__ w, Layout L, float gamma, DevScalars* sc)
{
    __shared__ unsigned long long red[2][NTHR / 32];
    unsigned long long m[2] = {0ull, 0ull};
    const long long n = (long long)L.nx * L.ny;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(v / L.nx), i = (int)(v % L.nx);
        float q[NF];
        for (int f = 0; f < NF; ++f) q[f] = w[L.idx(f, i, j, false)];
        float sx, sy;
        signal_speeds<float, false>(q[0], q[1], q[2], q[3], q[4], q[5], 0.f, 0.f, 0.f, 0.f, gamma, sx, sy);
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
        for (int k = 0; k < NTHR / 32; ++k) x = red[threadIdx.x][k] > x ? red[threadIdx.x][k] : x;
        atomicMax(&sc->cmax_bits[threadIdx.x], x);
    }
}

template <int CIN, int COUT>
constexpr size_t conv_smem() { return (size_t)(COUT * (9 * CIN + 8) + HH * HW * CIN) * 2; }
template <int CIN, int MO>
constexpr size_t dw_smem() { return (size_t)(HH * HW * CIN + TH * TW * MO) * 2; }

int grid_n(long long n, int cap) { long long g = (n + 255) / 256; return (int)(g < 1 ? 1 : (g > cap ? cap : g)); }

}  // namespace

struct sac_cnn {
    int H = 0, W = 0, device = 0, nsm = 148, conv_grid = 0;
    int tensor_path = 0;                // 0: mma.sync, 1: tcgen05 (cp.async halo), 2: tcgen05 (tensor-map halo)
    CUtensorMap tmaps[8];               // tensor maps of the convolution inputs (path 2)
    const void* tmap_ptr[8] = {nullptr};
    int tmap_c[8] = {0};
    int ntmap = 0;
    float clip = 0.f;                   // > 0: sac_cnn_apply limits the output to [-clip, clip]
    int positive = 0;                   // 1: no correction where it would halve density or pressure
    int* tc_err = nullptr;              // device flag: a tcgen05 accumulator wait gave up
    cudaStream_t stream = nullptr;
    float* params = nullptr;      // FP32 master [kParams]
    float* grads = nullptr;       // [kParams]
    float* adam_m = nullptr;
    float* adam_v = nullptr;
    long long adam_t = 0;
    __nv_bfloat16* wf[NLAYER] = {nullptr};
    __nv_bfloat16* wt[NLAYER] = {nullptr};
    float* bias[NLAYER] = {nullptr};
    __nv_bfloat16* feat = nullptr;      // [P][16]
    __nv_bfloat16* act[3] = {nullptr};  // [P][32]
    float* pred = nullptr;              // [P][8]
    __nv_bfloat16* dy3 = nullptr;       // [P][16]
    __nv_bfloat16* dact[3] = {nullptr}; // [P][32] gradients of act[0..2]
    float* part = nullptr;              // dW partials
    float* dbpart = nullptr;
    float* loss_part = nullptr;
    float* state = nullptr;             // packed FP32 [6][P] (for sac_cnn_apply)
    float* in_scale = nullptr;          // [8]
    float* out_scale = nullptr;         // [6]
    float h_loss_part[1024];
    char err[512] = {0};
};

static int cfail(sac_cnn* c, int code, const char* fmt, ...)
{
    if (c) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(c->err, sizeof(c->err), fmt, ap);
        va_end(ap);
    }
    return code;
}
#define CC(call)                                                                          \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return cfail(c, e_ == cudaErrorMemoryAllocation ? SAC_ERR_OOM : SAC_ERR_CUDA, \
                         "%s failed: %s", #call, cudaGetErrorString(e_));                 \
    } while (0)

// The convolutions run on the tcgen05 kernel (N = COUT rounded up to 16);
// the mma.sync kernel stays as the timed baseline (sac_cnn_set_tensor_path).
template <int CIN, int COUT, int MODE>
static cudaError_t run_conv(sac_cnn* c, const __nv_bfloat16* in, const __nv_bfloat16* w, const float* bias, void* out,
                            const __nv_bfloat16* mask)
{
    ConvArgs a;
    a.in = in; a.w = w; a.bias = bias; a.out = out; a.mask = mask; a.H = c->H; a.W = c->W;
    if (c->tensor_path == 2) {
        constexpr int NC = COUT < 16 ? 16 : COUT, RT = 2;
        const CUtensorMap* tm = nullptr;
        for (int k = 0; k < c->ntmap; ++k)
            if (c->tmap_ptr[k] == in && c->tmap_c[k] == CIN) tm = &c->tmaps[k];
        if (!tm) return cudaErrorInvalidValue;
        constexpr int bytes = tcv::TmaSmem<CIN, NC, RT>::BYTES;
        // resident CTAs per SM: as many as shared memory and the 512 tensor-memory columns allow
        constexpr int by_smem = (227 * 1024) / (bytes + 1024), by_tmem = 512 / tcv::TmaSmem<CIN, NC, RT>::TMEM_COLS;
        constexpr int per_sm = by_smem < by_tmem ? by_smem : by_tmem;
        const int tiles = ((c->W + tcv::TP - 1) / tcv::TP) * ((c->H + RT - 1) / RT);
        const int cap = per_sm * c->nsm;
        tcv::conv3x3_tma_kernel<CIN, COUT, NC, MODE, RT>
            <<<tiles < cap ? tiles : cap, tcv::NTHR_TC, bytes, c->stream>>>(a, *tm, c->tc_err);
    } else if (c->tensor_path == 1) {
        constexpr int NC = COUT < 16 ? 16 : COUT;
        // resident CTAs per SM: as many as shared memory and the 512 tensor-memory columns allow
        constexpr int by_smem = (227 * 1024) / (tcv::TcSmem<CIN, NC>::BYTES + 1024);
        constexpr int by_tmem = 512 / tcv::TcSmem<CIN, NC>::TMEM_COLS;
        constexpr int per_sm = by_smem < by_tmem ? by_smem : by_tmem;
        const int tiles = ((c->W + tcv::TP - 1) / tcv::TP) * ((c->H + tcv::ROWS - 1) / tcv::ROWS);
        const int cap = per_sm * c->nsm;
        const int grid = tiles < cap ? tiles : cap;
        tcv::conv3x3_tc_kernel<CIN, COUT, NC, MODE>
            <<<grid, tcv::NTHR_TC, tcv::TcSmem<CIN, NC>::BYTES, c->stream>>>(a, c->tc_err);
    } else {
        conv3x3_kernel<CIN, COUT, MODE><<<c->conv_grid, NTHR, conv_smem<CIN, COUT>(), c->stream>>>(a);
    }
    return cudaGetLastError();
}

template <int CIN, int MO>
static cudaError_t run_dw(sac_cnn* c, const __nv_bfloat16* dy, const __nv_bfloat16* x, int layer)
{
    DwArgs a;
    a.dy = dy; a.x = x; a.part = c->part; a.dbpart = c->dbpart; a.H = c->H; a.W = c->W;
    conv3x3_dw_kernel<CIN, MO><<<c->conv_grid, NTHR, dw_smem<CIN, MO>(), c->stream>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const long long off = param_offset(layer);
    const int cin = CIN_REAL[layer], cout = COUT_REAL[layer];
    dw_reduce_kernel<<<grid_n(cout * cin * 9 + cout, 1024), 256, 0, c->stream>>>(
        c->part, c->dbpart, c->conv_grid, CIN, MO, cin, cout, c->grads + off, c->grads + off + (long long)cout * cin * 9);
    return cudaGetLastError();
}

static cudaError_t pack_all(sac_cnn* c)
{
    for (int k = 0; k < NLAYER; ++k) {
        pack_weights_kernel<<<64, 256, 0, c->stream>>>(c->params + param_offset(k), CIN_REAL[k], COUT_REAL[k],
                                                       CIN_PAD[k], COUT_PAD[k], COUT_PAD[k] < 16 ? 16 : COUT_PAD[k],
                                                       c->wf[k], c->wt[k], c->bias[k]);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// features of the packed state -> forward through the 4 layers -> pred [P][8]
static cudaError_t forward_all(sac_cnn* c, const float* w, double gamma, double dx, double dy)
{
    const long long P = (long long)c->H * c->W;
    features_kernel<<<grid_n(P, 4096), 256, 0, c->stream>>>(w, c->H, c->W, (float)(gamma - 1.0),
                                                            (float)(1.0 / (12.0 * dx)), (float)(1.0 / (12.0 * dy)),
                                                            c->in_scale, c->feat);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = run_conv<16, 32, MODE_RELU>(c, c->feat, c->wf[0], c->bias[0], c->act[0], nullptr);
    if (e == cudaSuccess) e = run_conv<32, 32, MODE_RELU>(c, c->act[0], c->wf[1], c->bias[1], c->act[1], nullptr);
    if (e == cudaSuccess) e = run_conv<32, 32, MODE_RELU>(c, c->act[1], c->wf[2], c->bias[2], c->act[2], nullptr);
    if (e == cudaSuccess) e = run_conv<32, 8, MODE_LINEAR_F32>(c, c->act[2], c->wf[3], c->bias[3], c->pred, nullptr);
    return e;
}

// loss and gradients of every parameter into c->grads; *loss (host) if non-null
static int backward_all(sac_cnn* c, const float* w, const float* next, double* loss)
{
    const long long P = (long long)c->H * c->W;
    const int lg = 296;
    loss_kernel<<<lg, NTHR, 0, c->stream>>>(c->pred, w, next, c->out_scale, P, c->dy3, c->loss_part);
    CC(cudaGetLastError());
    CC((run_dw<32, 16>(c, c->dy3, c->act[2], 3)));
    CC((run_conv<16, 32, MODE_MASK>(c, c->dy3, c->wt[3], nullptr, c->dact[2], c->act[2])));
    CC((run_dw<32, 32>(c, c->dact[2], c->act[1], 2)));
    CC((run_conv<32, 32, MODE_MASK>(c, c->dact[2], c->wt[2], nullptr, c->dact[1], c->act[1])));
    CC((run_dw<32, 32>(c, c->dact[1], c->act[0], 1)));
    CC((run_conv<32, 32, MODE_MASK>(c, c->dact[1], c->wt[1], nullptr, c->dact[0], c->act[0])));
    CC((run_dw<16, 32>(c, c->dact[0], c->feat, 0)));
    if (loss) {
        CC(cudaMemcpyAsync(c->h_loss_part, c->loss_part, lg * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
        CC(cudaStreamSynchronize(c->stream));
        double s = 0.0;
        for (int k = 0; k < lg; ++k) s += c->h_loss_part[k];
        *loss = 0.5 * s / (6.0 * (double)P);
    }
    return SAC_OK;
}

template <int CIN, int COUT, int MODE>
static cudaError_t conv_attr()
{
    return cudaFuncSetAttribute(conv3x3_kernel<CIN, COUT, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)conv_smem<CIN, COUT>());
}
template <int CIN, int COUT, int NC, int MODE>
static cudaError_t tma_attr()
{
    return cudaFuncSetAttribute(tcv::conv3x3_tma_kernel<CIN, COUT, NC, MODE, 2>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tcv::TmaSmem<CIN, NC, 2>::BYTES);
}

// Tensor map of an NHWC BF16 image with C channels as the 4D tensor
// (8 channels, pixel, 8-channel chunk, row) and a box of (8, 130, C/8, 1): one
// copy lands one halo row in the [chunk][pixel][8 ch] layout of the tcgen05
// convolution (pixels left of 0 or right of W-1 read zeros).
static cudaError_t encode_nhwc_map(const void* img, int C, int W, int H, CUtensorMap* out)
{
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", (void**)&encode, 12000, cudaEnableDefault, &q) !=
                cudaSuccess || q != cudaDriverEntryPointSuccess || !encode)
            return cudaErrorNotSupported;
    }
    const cuuint64_t dims[4] = {8, (cuuint64_t)W, (cuuint64_t)(C / 8), (cuuint64_t)H};
    const cuuint64_t strides[3] = {(cuuint64_t)C * 2, 16, (cuuint64_t)W * C * 2};
    const cuuint32_t box[4] = {8, (cuuint32_t)tcv::HP, (cuuint32_t)(C / 8), 1};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    if (encode(out, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(img), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    return cudaSuccess;
}

template <int CIN, int COUT, int NC, int MODE>
static cudaError_t tc_attr()
{
    return cudaFuncSetAttribute(tcv::conv3x3_tc_kernel<CIN, COUT, NC, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)tcv::TcSmem<CIN, NC>::BYTES);
}
template <int CIN, int MO>
static cudaError_t dw_attr()
{
    return cudaFuncSetAttribute(conv3x3_dw_kernel<CIN, MO>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)dw_smem<CIN, MO>());
}

extern "C" {

long sac_cnn_param_count(void) { return (long)kParams; }

const char* sac_cnn_last_error(const sac_cnn* c) { return c ? c->err : "no network"; }

void sac_cnn_free(sac_cnn* c)
{
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    cudaFree(c->params); cudaFree(c->grads); cudaFree(c->adam_m); cudaFree(c->adam_v);
    for (int k = 0; k < NLAYER; ++k) { cudaFree(c->wf[k]); cudaFree(c->wt[k]); cudaFree(c->bias[k]); }
    cudaFree(c->feat); for (int k = 0; k < 3; ++k) { cudaFree(c->act[k]); cudaFree(c->dact[k]); }
    cudaFree(c->pred); cudaFree(c->dy3); cudaFree(c->part); cudaFree(c->dbpart); cudaFree(c->loss_part);
    cudaFree(c->state); cudaFree(c->in_scale); cudaFree(c->out_scale); cudaFree(c->tc_err);
    delete c;
}

int sac_cnn_init(int nx, int ny, int device, void* stream, sac_cnn** out)
{
    if (out) *out = nullptr;
    if (!out || nx < 8 || ny < 8 || nx > 16384 || ny > 16384) return SAC_ERR_ARG;
    sac_cnn* c = new sac_cnn();
    c->H = ny; c->W = nx; c->device = device; c->stream = (cudaStream_t)stream;
    int rc = SAC_OK;
    do {
        if (cudaSetDevice(device) != cudaSuccess) { rc = cfail(c, SAC_ERR_ARG, "device %d", device); break; }
        cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, device);
        c->conv_grid = 4 * c->nsm;
        const long long P = (long long)nx * ny;
        bool ok = true;
        auto A = [&](void** p, size_t bytes) { if (ok && cudaMalloc(p, bytes) != cudaSuccess) ok = false; if (ok) cudaMemset(*p, 0, bytes); };
        A((void**)&c->params, kParams * 4); A((void**)&c->grads, kParams * 4);
        A((void**)&c->adam_m, kParams * 4); A((void**)&c->adam_v, kParams * 4);
        for (int k = 0; k < NLAYER; ++k) {
            const size_t nwp = (size_t)COUT_PAD[k] * 9 * CIN_PAD[k];
            A((void**)&c->wf[k], nwp * 2);
            A((void**)&c->wt[k], (size_t)CIN_PAD[k] * 9 * (COUT_PAD[k] < 16 ? 16 : COUT_PAD[k]) * 2);
            A((void**)&c->bias[k], COUT_PAD[k] * 4);
        }
        A((void**)&c->feat, P * 16 * 2);
        for (int k = 0; k < 3; ++k) { A((void**)&c->act[k], P * 32 * 2); A((void**)&c->dact[k], P * 32 * 2); }
        A((void**)&c->pred, P * 8 * 4); A((void**)&c->dy3, P * 16 * 2);
        A((void**)&c->part, (size_t)c->conv_grid * 32 * 9 * 32 * 4); A((void**)&c->dbpart, (size_t)c->conv_grid * 32 * 4);
        A((void**)&c->loss_part, 1024 * 4);
        A((void**)&c->state, P * NF * 4);
        A((void**)&c->in_scale, 8 * 4); A((void**)&c->out_scale, 6 * 4);
        A((void**)&c->tc_err, 4);
        if (!ok) { rc = cfail(c, SAC_ERR_OOM, "network buffers"); break; }
        cudaError_t e = conv_attr<16, 32, MODE_RELU>();
        if (e == cudaSuccess) e = conv_attr<32, 32, MODE_RELU>();
        if (e == cudaSuccess) e = conv_attr<32, 8, MODE_LINEAR_F32>();
        if (e == cudaSuccess) e = conv_attr<16, 32, MODE_MASK>();
        if (e == cudaSuccess) e = conv_attr<32, 32, MODE_MASK>();
        if (e == cudaSuccess) e = dw_attr<32, 16>();
        if (e == cudaSuccess) e = dw_attr<32, 32>();
        if (e == cudaSuccess) e = dw_attr<16, 32>();
        if (e == cudaSuccess) e = tc_attr<16, 32, 32, MODE_RELU>();
        if (e == cudaSuccess) e = tc_attr<32, 32, 32, MODE_RELU>();
        if (e == cudaSuccess) e = tc_attr<32, 8, 16, MODE_LINEAR_F32>();
        if (e == cudaSuccess) e = tc_attr<16, 32, 32, MODE_MASK>();
        if (e == cudaSuccess) e = tc_attr<32, 32, 32, MODE_MASK>();
        if (e == cudaSuccess) e = tma_attr<16, 32, 32, MODE_RELU>();
        if (e == cudaSuccess) e = tma_attr<32, 32, 32, MODE_RELU>();
        if (e == cudaSuccess) e = tma_attr<32, 8, 16, MODE_LINEAR_F32>();
        if (e == cudaSuccess) e = tma_attr<16, 32, 32, MODE_MASK>();
        if (e == cudaSuccess) e = tma_attr<32, 32, 32, MODE_MASK>();
        if (e == cudaSuccess) {
            // the convolution inputs: features, the three hidden activations, the output
            // gradient and the two hidden input gradients the backward pass convolves
            const void* img[7] = {c->feat, c->act[0], c->act[1], c->act[2], c->dy3, c->dact[2], c->dact[1]};
            const int ch[7] = {16, 32, 32, 32, 16, 32, 32};
            c->ntmap = 0;
            for (int k = 0; k < 7; ++k)
                if (encode_nhwc_map(img[k], ch[k], nx, ny, &c->tmaps[c->ntmap]) == cudaSuccess) {
                    c->tmap_ptr[c->ntmap] = img[k];
                    c->tmap_c[c->ntmap++] = ch[k];
                }
            cudaGetLastError();
        }
        if (e != cudaSuccess) { rc = cfail(c, SAC_ERR_CUDA, "kernel set-up: %s", cudaGetErrorString(e)); break; }
        const float ones[8] = {1, 1, 1, 1, 1, 1, 1, 1};
        if (cudaMemcpy(c->in_scale, ones, 32, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(c->out_scale, ones, 24, cudaMemcpyHostToDevice) != cudaSuccess) {
            rc = cfail(c, SAC_ERR_CUDA, "scales"); break;
        }
    } while (0);
    if (rc != SAC_OK) { sac_cnn_free(c); return rc; }
    *out = c;
    return SAC_OK;
}

int sac_cnn_set_tensor_path(sac_cnn* c, int path)
{
    if (!c || path < 0 || path > 2) return SAC_ERR_ARG;
    if (path == 2 && c->ntmap < 7) return cfail(c, SAC_ERR_CUDA, "tensor maps of the activations could not be encoded");
    CC(cudaSetDevice(c->device));
    CC(cudaStreamSynchronize(c->stream));
    c->tensor_path = path;
    return SAC_OK;
}

int sac_cnn_set_limiter(sac_cnn* c, double clip, int keep_positive)
{
    if (!c || !(clip >= 0.0) || !std::isfinite(clip) || (keep_positive != 0 && keep_positive != 1)) return SAC_ERR_ARG;
    c->clip = (float)clip;
    c->positive = keep_positive;
    return SAC_OK;
}

int sac_cnn_sync(sac_cnn* c)
{
    if (!c) return SAC_ERR_ARG;
    CC(cudaSetDevice(c->device));
    int h = 0;
    CC(cudaMemcpyAsync(&h, c->tc_err, 4, cudaMemcpyDeviceToHost, c->stream));
    CC(cudaStreamSynchronize(c->stream));
    if (h) {
        CC(cudaMemsetAsync(c->tc_err, 0, 4, c->stream));
        return cfail(c, SAC_ERR_TIMEOUT, "a tensor-core accumulator wait gave up");
    }
    return SAC_OK;
}

int sac_cnn_set_params(sac_cnn* c, const float* params, long n)
{
    if (!c || !params || n != (long)kParams) return cfail(c, SAC_ERR_ARG, "expected %lld parameters", kParams);
    CC(cudaSetDevice(c->device));
    CC(cudaMemcpyAsync(c->params, params, kParams * 4, cudaMemcpyHostToDevice, c->stream));
    CC(cudaMemsetAsync(c->adam_m, 0, kParams * 4, c->stream));
    CC(cudaMemsetAsync(c->adam_v, 0, kParams * 4, c->stream));
    c->adam_t = 0;
    CC(pack_all(c));
    CC(cudaStreamSynchronize(c->stream));
    return SAC_OK;
}

int sac_cnn_get_params(sac_cnn* c, float* params, long n)
{
    if (!c || !params || n != (long)kParams) return cfail(c, SAC_ERR_ARG, "expected %lld parameters", kParams);
    CC(cudaSetDevice(c->device));
    CC(cudaMemcpyAsync(params, c->params, kParams * 4, cudaMemcpyDeviceToHost, c->stream));
    CC(cudaStreamSynchronize(c->stream));
    return SAC_OK;
}

int sac_cnn_set_scales(sac_cnn* c, const float in_scale[8], const float out_scale[6])
{
    if (!c || !in_scale || !out_scale) return SAC_ERR_ARG;
    CC(cudaSetDevice(c->device));
    CC(cudaMemcpyAsync(c->in_scale, in_scale, 32, cudaMemcpyHostToDevice, c->stream));
    CC(cudaMemcpyAsync(c->out_scale, out_scale, 24, cudaMemcpyHostToDevice, c->stream));
    CC(cudaStreamSynchronize(c->stream));
    return SAC_OK;
}

int sac_cnn_forward(sac_cnn* c, const float* w, double gamma, double dx, double dy, float* pred)
{
    if (!c || !w || !pred) return SAC_ERR_ARG;
    CC(cudaSetDevice(c->device));
    CC(forward_all(c, w, gamma, dx, dy));
    CC(cudaMemcpyAsync(pred, c->pred, (size_t)c->H * c->W * 8 * 4, cudaMemcpyDeviceToDevice, c->stream));
    return SAC_OK;
}

int sac_cnn_grads(sac_cnn* c, const float* w, const float* next, double gamma, double dx, double dy,
                  float* grads, double* loss)
{
    if (!c || !w || !next) return SAC_ERR_ARG;
    CC(cudaSetDevice(c->device));
    CC(forward_all(c, w, gamma, dx, dy));
    int rc = backward_all(c, w, next, loss);
    if (rc != SAC_OK) return rc;
    if (grads) {
        CC(cudaMemcpyAsync(grads, c->grads, kParams * 4, cudaMemcpyDeviceToHost, c->stream));
        CC(cudaStreamSynchronize(c->stream));
    }
    return SAC_OK;
}

int sac_cnn_train_step(sac_cnn* c, const float* w, const float* next, double gamma, double dx, double dy,
                       double lr, double* loss)
{
    if (!c || !w || !next || !(lr > 0.0)) return SAC_ERR_ARG;
    CC(cudaSetDevice(c->device));
    CC(forward_all(c, w, gamma, dx, dy));
    int rc = backward_all(c, w, next, loss);
    if (rc != SAC_OK) return rc;
    c->adam_t += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = (float)(1.0 - std::pow(0.9, (double)c->adam_t)), c2 = (float)(1.0 - std::pow(0.999, (double)c->adam_t));
    adam_kernel<<<grid_n(kParams, 256), 256, 0, c->stream>>>(c->params, c->grads, c->adam_m, c->adam_v, kParams,
                                                             (float)lr, b1, b2, 1e-8f, c1, c2);
    CC(cudaGetLastError());
    CC(pack_all(c));
    return SAC_OK;
}

int sac_cnn_apply(sac_ctx* ctx, sac_cnn* c)
{
    if (!ctx || !c) return SAC_ERR_ARG;
    if (!ctx->fp32 || ctx->p.has_background || ctx->p.bc_x != SAC_BC_PERIODIC || ctx->p.bc_y != SAC_BC_PERIODIC ||
        ctx->p.nx != c->W || ctx->p.ny != c->H)
        return cfail(c, SAC_ERR_ARG, "the correction needs a periodic FP32 run of the network's size");
    if (!ctx->have_state) return cfail(c, SAC_ERR_STATE, "no state");
    CC(cudaSetDevice(c->device));
    const long long P = (long long)c->H * c->W;
    float* u0 = (float*)ctx->u0;
    export_paired_kernel<<<grid_n(P * 3, 4096), 256, 0, c->stream>>>(u0, ctx->L, c->state);
    CC(cudaGetLastError());
    CC(forward_all(c, c->state, ctx->p.gamma, ctx->dx, ctx->dy));
    const int nsum = 148;
    const float gm1 = (float)(ctx->p.gamma - 1.0);
    pred_sum_kernel<<<nsum, NTHR, 0, c->stream>>>(c->pred, P, c->clip, c->state, c->out_scale, gm1, c->positive,
                                                  c->loss_part);
    CC(cudaGetLastError());
    const long long ng = (long long)(ctx->p.nx + 2 * GY) * (ctx->p.ny + 2 * GY);
    add_correction_kernel<<<grid_n(ng, 4096), 256, 0, c->stream>>>(u0, ctx->L, c->pred, c->out_scale, c->loss_part,
                                                                   nsum, c->clip, c->state, gm1, c->positive, ctx->sc);
    CC(cudaGetLastError());
    cmax_paired_kernel<<<grid_n(P, 2048), NTHR, 0, c->stream>>>(u0, ctx->L, (float)ctx->p.gamma, ctx->sc);
    CC(cudaGetLastError());
    return SAC_OK;
}

int sac_cnn_perturb(sac_cnn* c, const float* w, float* out, const float amp[6], unsigned long long seed)
{
    if (!c || !w || !out || !amp) return SAC_ERR_ARG;
    CC(cudaSetDevice(c->device));
    CC(cudaMemcpyAsync(c->loss_part + 1000, amp, 6 * sizeof(float), cudaMemcpyHostToDevice, c->stream));
    const long long n = (long long)c->H * c->W;
    perturb_kernel<<<grid_n(n * NF, 4096), 256, 0, c->stream>>>(w, out, n, c->loss_part + 1000, seed);
    CC(cudaGetLastError());
    CC(cudaStreamSynchronize(c->stream));
    return SAC_OK;
}

int sac_block_average(const float* fine, int nfields, int nxf, int nyf, int r, float* coarse, void* stream)
{
    if (!fine || !coarse || nfields < 1 || r < 1 || nxf % r || nyf % r) return SAC_ERR_ARG;
    const long long n = (long long)nfields * (nxf / r) * (nyf / r);
    block_average_kernel<<<grid_n(n, 4096), 256, 0, (cudaStream_t)stream>>>(fine, nfields, nyf, nxf, r, coarse);
    return cudaGetLastError() == cudaSuccess ? SAC_OK : SAC_ERR_CUDA;
}

}  // extern "C"
