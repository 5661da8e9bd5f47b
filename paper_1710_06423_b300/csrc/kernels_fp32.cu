// kernels_fp32.cu -- launchers of the FP32 fused RK stage kernel (field-pair
// layout, packed f32x2 arithmetic, D-scheme RK registers).
#include <algorithm>
#include <cstring>
#include <mutex>

#include <cudaTypedefs.h>

#include "stage_fp32.cuh"

namespace sac {
namespace {
using f32k::NT;
using f32k::TX;
using f32k::TY;

template <int S, bool BG, bool HD, bool GR, bool SF>
cudaError_t set_attr()
{
    cudaError_t e = cudaFuncSetAttribute(f32k::stage_fp32<S, BG, HD, GR, SF>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(f32k::Smem));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(f32k::stage_fp32<S, BG, HD, GR, SF>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 cudaSharedmemCarveoutMaxShared);
    return e;
}

int g_resident = 296;   // persistent grid: resident CTAs on the device (2 per SM)

// Tensor maps of the stage inputs (3D: pitch float2 x padded rows x 3 planes;
// box RXP x RY x 1), encoded once per buffer and layout (the CUDA driver API's encoder
// is reached through the runtime's entry-point query: no link to libcuda).
struct TmEntry {
    const void* p;
    int pitch, rows;
    long long fstride;
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
        if (g_tm[i].p == a.sin && g_tm[i].pitch == a.L.pitch && g_tm[i].rows == a.L.rows && g_tm[i].fstride == a.L.fstride) {
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
    const cuuint32_t box[3] = {(cuuint32_t)f32k::RXP, (cuuint32_t)f32k::RY, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    CUtensorMap tm;
    if (encode(&tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3, const_cast<float*>(a.sin), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    TmEntry& e = g_ntm < 16 ? g_tm[g_ntm++] : g_tm[(g_tm_next++) % 16];
    e = TmEntry{a.sin, a.L.pitch, a.L.rows, a.L.fstride, tm};
    *out = tm;
    return cudaSuccess;
}

namespace {

__global__ void halo_fp32(const StageArgs<float> a, long long n)
{
    if (a.sc->skip) return;
    float2* w = reinterpret_cast<float2*>(a.sout);
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
        f32k::halo_cell(w, a.L, a.bc_x, a.bc_y, t);
}

template <int S, bool BG, bool HD, bool GR, bool SF>
cudaError_t launch(const StageArgs<float>& a, cudaStream_t s)
{
    const int ntx = (a.L.nx + TX - 1) / TX, nty = (a.L.ny + TY - 1) / TY, ntiles = ntx * nty;
    const int grid = ntiles < g_resident ? ntiles : g_resident;
    CUtensorMap tm;
    const cudaError_t te = encode_stage_tensor_map(a, &tm);
    if (te != cudaSuccess) return te;
    f32k::stage_fp32<S, BG, HD, GR, SF><<<grid, NT, sizeof(f32k::Smem), s>>>(a, ntx, ntiles, tm);
    if (a.bc_x != BC_FIXED || a.bc_y != BC_FIXED) {
        const long long n = f32k::halo_count(a.L);
        const int hb = (int)std::min<long long>((n + 255) / 256, g_resident * 2);
        halo_fp32<<<hb, 256, 0, s>>>(a, n);
    }
    return cudaGetLastError();
}

template <bool BG, bool HD, bool GR = false, bool SF = false>
cudaError_t by_stage(const StageArgs<float>& a, int stage, cudaStream_t s)
{
    switch (stage) {
        case 1: return launch<1, BG, HD, GR, SF>(a, s);
        case 2: return launch<2, BG, HD, GR, SF>(a, s);
        case 3: return launch<3, BG, HD, GR, SF>(a, s);
        default: return launch<4, BG, HD, GR, SF>(a, s);
    }
}

template <bool BG, bool HD, bool GR = false, bool SF = false>
cudaError_t attr_all()
{
    cudaError_t e = set_attr<1, BG, HD, GR, SF>();
    if (e == cudaSuccess) e = set_attr<2, BG, HD, GR, SF>();
    if (e == cudaSuccess) e = set_attr<3, BG, HD, GR, SF>();
    if (e == cudaSuccess) e = set_attr<4, BG, HD, GR, SF>();
    return e;
}
}  // namespace

cudaError_t prepare_stage_fp32()
{
    int dev = 0, nsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    g_resident = 2 * nsm;
    e = attr_all<false, false>();
    if (e == cudaSuccess) e = attr_all<false, true>();
    if (e == cudaSuccess) e = attr_all<true, false>();
    if (e == cudaSuccess) e = attr_all<true, true>();
    if (e == cudaSuccess) e = attr_all<true, false, true>();
    if (e == cudaSuccess) e = attr_all<true, true, true>();
    if (e == cudaSuccess) e = attr_all<false, true, false, true>();
    return e;
}

cudaError_t launch_stage_fp32(const StageArgs<float>& a, int stage, bool hd, bool bg, cudaStream_t s)
{
    // the single-face variant: no background, no gravity (checked by sac_init)
    if (a.hd_single_face && hd) return by_stage<false, true, false, true>(a, stage, s);
    // gravity needs a background (checked by sac_init)
    if (bg && a.has_grav())
        return hd ? by_stage<true, true, true>(a, stage, s) : by_stage<true, false, true>(a, stage, s);
    if (bg) return hd ? by_stage<true, true>(a, stage, s) : by_stage<true, false>(a, stage, s);
    return hd ? by_stage<false, true>(a, stage, s) : by_stage<false, false>(a, stage, s);
}

}  // namespace sac
