// kernels_fp32.cu -- launchers of the FP32 fused RK stage kernel (field-pair
// layout, packed f32x2 arithmetic, D-scheme RK registers).
#include <algorithm>
#include <cstring>
#include <mutex>

#include <cudaTypedefs.h>

#include "stage_fp32.cuh"

namespace sac {
namespace {

template <class G, int S, bool BG, bool HD, bool GR, bool SF, bool KG = false>
cudaError_t set_attr()
{
    cudaError_t e = cudaFuncSetAttribute(f32k::stage_fp32<G, S, BG, HD, GR, SF, KG>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(f32k::Smem<G>));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(f32k::stage_fp32<G, S, BG, HD, GR, SF, KG>,
                                 cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    return e;
}

int g_nsm = 148;   // SMs of the device (persistent grids: resident CTAs per SM x this)

// Tensor maps of the stage inputs (3D: pitch float2 x padded rows x 3 planes;
// box RXP x RY x 1), encoded once per buffer and layout (the CUDA driver API's encoder
// is reached through the runtime's entry-point query: no link to libcuda).
struct TmEntry {
    const void* p;
    int pitch, rows;
    long long fstride;
    int tile;
    CUtensorMap tm;
};
TmEntry g_tm[16];
int g_ntm = 0, g_tm_next = 0;
std::mutex g_tm_mu;
}  // namespace

cudaError_t encode_stage_tensor_map(const StageArgs<float>& a, CUtensorMap* out)
{
    std::lock_guard<std::mutex> lk(g_tm_mu);
    for (int i = 0; i < g_ntm; ++i)
        if (g_tm[i].p == a.sin && g_tm[i].pitch == a.L.pitch && g_tm[i].rows == a.L.rows &&
            g_tm[i].fstride == a.L.fstride && g_tm[i].tile == a.tile) {
            *out = g_tm[i].tm;
            return cudaSuccess;
        }
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", (void**)&encode, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !encode)
            return cudaErrorNotSupported;
    }
    const cuuint64_t dims[3] = {(cuuint64_t)a.L.pitch, (cuuint64_t)a.L.rows, 3};
    const cuuint64_t strides[2] = {(cuuint64_t)a.L.pitch * sizeof(float2), (cuuint64_t)a.L.fstride * sizeof(float2)};
    const int bx = a.tile == TILE_64x16 ? f32k::G64x16::RXP : (a.tile == TILE_32x16 ? f32k::G32x16::RXP : f32k::G32x32::RXP);
    const int by = a.tile == TILE_64x16 ? f32k::G64x16::RY : (a.tile == TILE_32x16 ? f32k::G32x16::RY : f32k::G32x32::RY);
    const cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    CUtensorMap tm;
    if (encode(&tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3, const_cast<float*>(a.sin), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    TmEntry& e = g_ntm < 16 ? g_tm[g_ntm++] : g_tm[(g_tm_next++) % 16];
    e = TmEntry{a.sin, a.L.pitch, a.L.rows, a.L.fstride, a.tile, tm};
    *out = tm;
    return cudaSuccess;
}

namespace {

__global__ void halo_fp32(const StageArgs<float> a, long long n)
{
    pdl_launch_dependents();
    pdl_wait();
    if (a.sc->skip) return;
    float2* w = reinterpret_cast<float2*>(a.sout);
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
        f32k::halo_cell(w, a.L, a.bc_x, a.bc_y, t);
}

template <class G, int S, bool BG, bool HD, bool GR, bool SF, bool KG>
cudaError_t launch(const StageArgs<float>& a, cudaStream_t s)
{
    const int ntx = (a.L.nx + G::TX - 1) / G::TX, nty = (a.L.ny + G::TY - 1) / G::TY, ntiles = ntx * nty;
    const int resident = G::MINB * g_nsm;
    const int grid = ntiles < resident ? ntiles : resident;
    CUtensorMap tm;
    const cudaError_t te = encode_stage_tensor_map(a, &tm);
    if (te != cudaSuccess) return te;
    // both kernels may be scheduled while their predecessor runs (see pdl_wait)
    cudaError_t e = launch_pdl(f32k::stage_fp32<G, S, BG, HD, GR, SF, KG>, dim3(grid), dim3(G::NT),
                               sizeof(f32k::Smem<G>), s, a, ntx, ntiles, tm);
    if (!KG && e == cudaSuccess && (a.bc_x != BC_FIXED || a.bc_y != BC_FIXED)) {
        const long long n = f32k::halo_count(a.L);
        const int hb = (int)std::min<long long>((n + 255) / 256, 4 * g_nsm);
        e = launch_pdl(halo_fp32, dim3(hb), dim3(256), 0, s, a, n);
    }
    return e;
}

template <class G, bool BG, bool HD, bool GR = false, bool SF = false, bool KG = false>
cudaError_t by_stage(const StageArgs<float>& a, int stage, cudaStream_t s)
{
    switch (stage) {
        case 1: return launch<G, 1, BG, HD, GR, SF, KG>(a, s);
        case 2: return launch<G, 2, BG, HD, GR, SF, KG>(a, s);
        case 3: return launch<G, 3, BG, HD, GR, SF, KG>(a, s);
        default: return launch<G, 4, BG, HD, GR, SF, KG>(a, s);
    }
}

// the tile shapes are instantiated for the plain and background variants, the
// in-kernel ghost frame for the plain variants only (a background run ignores
// it); the gravity and single-face variants run 32 x 32 tiles
template <class G, bool BG, bool HD>
cudaError_t by_ghosts(const StageArgs<float>& a, int stage, cudaStream_t s)
{
    if constexpr (!BG) {
        if (a.kernel_ghosts) return by_stage<G, BG, HD, false, false, true>(a, stage, s);
    }
    return by_stage<G, BG, HD>(a, stage, s);
}
template <bool BG, bool HD>
cudaError_t by_tile(const StageArgs<float>& a, int stage, cudaStream_t s)
{
    switch (a.tile) {
        case TILE_64x16: return by_ghosts<f32k::G64x16, BG, HD>(a, stage, s);
        case TILE_32x16: return by_ghosts<f32k::G32x16, BG, HD>(a, stage, s);
        default: return by_ghosts<f32k::G32x32, BG, HD>(a, stage, s);
    }
}

template <class G, bool BG, bool HD, bool GR = false, bool SF = false, bool KG = false>
cudaError_t attr_all()
{
    cudaError_t e = set_attr<G, 1, BG, HD, GR, SF, KG>();
    if (e == cudaSuccess) e = set_attr<G, 2, BG, HD, GR, SF, KG>();
    if (e == cudaSuccess) e = set_attr<G, 3, BG, HD, GR, SF, KG>();
    if (e == cudaSuccess) e = set_attr<G, 4, BG, HD, GR, SF, KG>();
    return e;
}
template <class G>
cudaError_t attr_geometry()
{
    cudaError_t e = attr_all<G, false, false>();
    if (e == cudaSuccess) e = attr_all<G, false, true>();
    if (e == cudaSuccess) e = attr_all<G, true, false>();
    if (e == cudaSuccess) e = attr_all<G, true, true>();
    if (e == cudaSuccess) e = attr_all<G, false, false, false, false, true>();
    if (e == cudaSuccess) e = attr_all<G, false, true, false, false, true>();
    return e;
}
}  // namespace

cudaError_t prepare_stage_fp32()
{
    int dev = 0, nsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    g_nsm = nsm;
    e = attr_geometry<f32k::G32x32>();
    if (e == cudaSuccess) e = attr_geometry<f32k::G64x16>();
    if (e == cudaSuccess) e = attr_geometry<f32k::G32x16>();
    if (e == cudaSuccess) e = attr_all<f32k::G32x32, true, false, true>();
    if (e == cudaSuccess) e = attr_all<f32k::G32x32, true, true, true>();
    if (e == cudaSuccess) e = attr_all<f32k::G32x32, false, true, false, true>();
    return e;
}

cudaError_t launch_stage_fp32(const StageArgs<float>& a, int stage, bool hd, bool bg, cudaStream_t s)
{
    using f32k::G32x32;
    if ((a.hd_single_face && hd) || (bg && a.has_grav())) {
        StageArgs<float> b = a;   // these variants run 32 x 32 tiles whatever the context's shape
        b.tile = TILE_32x32;
        // the single-face variant: no background, no gravity (checked by sac_init)
        if (b.hd_single_face && hd) return by_stage<G32x32, false, true, false, true>(b, stage, s);
        // gravity needs a background (checked by sac_init)
        return hd ? by_stage<G32x32, true, true, true>(b, stage, s) : by_stage<G32x32, true, false, true>(b, stage, s);
    }
    if (bg) return hd ? by_tile<true, true>(a, stage, s) : by_tile<true, false>(a, stage, s);
    return hd ? by_tile<false, true>(a, stage, s) : by_tile<false, false>(a, stage, s);
}

}  // namespace sac
