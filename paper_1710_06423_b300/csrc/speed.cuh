// speed.cuh -- maximum signal speed of one cell, |v_d| + c_fast with
// c_fast^2 = (gamma p_k + |B|^2) / rho (total p_k, total B), the quantity whose
// grid-wide maximum sets the CFL step and scales the hyper-diffusion
// (section 2 of arXiv 1710.06423).
//
// Written with explicit round-to-nearest intrinsics so that no FMA is ever
// contracted into it: the fused stage-4 reduction and the stand-alone
// reduction after a state import (different translation units, different
// contraction settings) produce the same bits, and a resumed run takes the
// same steps as an uninterrupted one.
#pragma once
#include <cuda_runtime.h>

namespace sac {

struct RnF {
    using T = float;
    static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
    static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
    static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
    static __device__ __forceinline__ float div(float a, float b) { return __fdiv_rn(a, b); }
    static __device__ __forceinline__ float sqrt_(float a) { return __fsqrt_rn(a); }
    static __device__ __forceinline__ float abs_(float a) { return fabsf(a); }
};
struct RnD {
    using T = double;
    static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
    static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
    static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
    static __device__ __forceinline__ double div(double a, double b) { return __ddiv_rn(a, b); }
    static __device__ __forceinline__ double sqrt_(double a) { return __dsqrt_rn(a); }
    static __device__ __forceinline__ double abs_(double a) { return fabs(a); }
};
template <typename T> struct Rn;
template <> struct Rn<float> : RnF {};
template <> struct Rn<double> : RnD {};

// Conserved perturbations (rt, mx, my, et, btx, bty), background (rb, eb, bbx,
// bby; ignored when !BG) -> signal speeds along x and y.
// FP32: one reciprocal of rho and a square root, both the fixed approximate
// PTX instructions (relative error ~1e-7, far below what a CFL step needs),
// every other operation round-to-nearest.  Deterministic like the FP64 form,
// so every FP32 reduction (fused or stand-alone) gives the same bits.
template <bool BG>
__device__ __forceinline__ void signal_speeds_f32(float rt, float mx, float my, float et, float btx, float bty,
                                                  float rb, float eb, float bbx, float bby, float gamma,
                                                  float& sx, float& sy)
{
    using R = RnF;
    const float gm1 = R::sub(gamma, 1.f), half = 0.5f;
    float rho, pkt, bx, by;
    if constexpr (BG) rho = R::add(rb, rt); else rho = rt;
    float rinv;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rinv) : "f"(rho));
    const float ux = R::mul(mx, rinv), uy = R::mul(my, rinv);
    const float ekin = R::mul(half, R::add(R::mul(mx, ux), R::mul(my, uy)));
    const float b2p = R::mul(half, R::add(R::mul(btx, btx), R::mul(bty, bty)));
    if constexpr (BG) {
        const float bb = R::add(R::mul(bbx, btx), R::mul(bby, bty));
        const float pk = R::mul(gm1, R::sub(R::sub(R::sub(et, ekin), bb), b2p));
        const float b2b = R::mul(half, R::add(R::mul(bbx, bbx), R::mul(bby, bby)));
        pkt = R::add(R::mul(gm1, R::sub(eb, b2b)), pk);
        bx = R::add(bbx, btx); by = R::add(bby, bty);
    } else {
        pkt = R::mul(gm1, R::sub(R::sub(et, ekin), b2p));
        bx = btx; by = bty;
        (void)eb;
    }
    const float c2 = R::mul(R::add(R::mul(gamma, pkt), R::add(R::mul(bx, bx), R::mul(by, by))), rinv);
    float cf;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(cf) : "f"(c2));
    sx = R::add(fabsf(ux), cf);
    sy = R::add(fabsf(uy), cf);
}

template <typename T, bool BG>
__device__ __forceinline__ void signal_speeds(T rt, T mx, T my, T et, T btx, T bty,
                                              T rb, T eb, T bbx, T bby, T gamma,
                                              T& sx, T& sy)
{
    if constexpr (sizeof(T) == sizeof(float)) {
        signal_speeds_f32<BG>(rt, mx, my, et, btx, bty, rb, eb, bbx, bby, gamma, sx, sy);
        return;
    } else {
    using R = Rn<T>;
    const T gm1 = R::sub(gamma, (T)1), half = (T)0.5;
    T rho, ux, uy, pkt, bx, by;
    if constexpr (BG) {
        rho = R::add(rb, rt);
        ux = R::div(mx, rho); uy = R::div(my, rho);
        T ekin = R::mul(half, R::add(R::mul(mx, ux), R::mul(my, uy)));
        T bb = R::add(R::mul(bbx, btx), R::mul(bby, bty));
        T b2p = R::mul(half, R::add(R::mul(btx, btx), R::mul(bty, bty)));
        T pk = R::mul(gm1, R::sub(R::sub(R::sub(et, ekin), bb), b2p));
        T b2b = R::mul(half, R::add(R::mul(bbx, bbx), R::mul(bby, bby)));
        T pkb = R::mul(gm1, R::sub(eb, b2b));
        pkt = R::add(pkb, pk);
        bx = R::add(bbx, btx); by = R::add(bby, bty);
    } else {
        rho = rt;
        ux = R::div(mx, rho); uy = R::div(my, rho);
        T ekin = R::mul(half, R::add(R::mul(mx, ux), R::mul(my, uy)));
        T b2p = R::mul(half, R::add(R::mul(btx, btx), R::mul(bty, bty)));
        pkt = R::mul(gm1, R::sub(R::sub(et, ekin), b2p));
        bx = btx; by = bty;
        (void)rb; (void)eb; (void)bbx; (void)bby;
    }
    T cf = R::sqrt_(R::div(R::add(R::mul(gamma, pkt), R::add(R::mul(bx, bx), R::mul(by, by))), rho));
    sx = R::add(R::abs_(ux), cf);
    sy = R::add(R::abs_(uy), cf);
    }
}

__device__ __forceinline__ unsigned long long speed_key(double v) { return (unsigned long long)__double_as_longlong(v); }
__device__ __forceinline__ unsigned long long speed_key(float v) { return (unsigned long long)__float_as_uint(v); }

}  // namespace sac
