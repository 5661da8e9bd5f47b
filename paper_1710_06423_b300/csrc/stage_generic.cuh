// stage_generic.cuh -- one fused RK stage of the split ideal-MHD system
// (section 2 of arXiv 1710.06423), generic over the arithmetic type.
//
// One CTA owns a TX x TY tile of cells.  It stages the tile plus a 3-cell
// halo (4 columns on the left for 16-byte alignment) of the six conserved
// fields, and the two background field components, in shared memory, then:
//   1. primitives per staged cell: v = m/rho, perturbed total pressure,
//      energy-flux factor and B.v (section 2 pressure definitions);
//   2. shock indicator s = max(0, -div v) around the tile;
//   3. per conserved variable: ideal fluxes on the +-2 cross, face
//      hyper-diffusion fluxes nu d1 on the tile's faces, then
//      k = (H_x + H_y) - (D_x F_x + D_y F_y) per cell (fourth-order central
//      differences, section 2);
//   4. the RK stage update (classical RK4), the stage output with its ghost
//      copies, and in stage 4 the maximum signal speed of the new state,
//      reduced warp -> block -> one atomicMax per CTA.
//
// Every expression is written in the same order as the FP64 reference
// discretisation it implements, so the FP64 instantiation (compiled without
// FMA contraction) reproduces it to the last bit.
#pragma once
#include "sac_internal.cuh"
#include "speed.cuh"

namespace sac {

// RK register schemes (classical RK4, section 2), chosen per precision.
//  K (FP64; bit-compatible with U0 + dt/6 (((k1+2k2)+2k3)+k4)):
//    s1: K = k1,      S = U0 + dt/2 k1      s2: K += 2 k2, S = U0 + dt/2 k2
//    s3: K += 2 k3,   S = U0 + dt k3        s4: U0 = U0 + dt/6 (K + k4)
//    25.5 values moved per cell-stage.
//  A (accumulator of the new state; 21 values per cell-stage):
//    s1: S1 = U0 + dt/2 k1
//    s2: A = U0 + (S1 - U0)/3 + dt/3 k2,   S2 = U0 + dt/2 k2
//    s3: A += dt/3 k3,                     S3 = U0 + dt k3
//    s4: U0 = A + dt/6 k4
//  D (accumulator of the increment; 22.5 values per cell-stage):
//    s1: S1 = U0 + dt/2 k1
//    s2: D = (S1 - U0)/3 + dt/3 k2,        S2 = U0 + dt/2 k2
//    s3: D += dt/3 k3,                     S3 = U0 + dt k3
//    s4: U0 = U0 + (D + dt/6 k4)
//    S1 - U0 is exact when the two are within a factor of two (Sterbenz), so
//    D carries dt/6 k1 without the rounding of a state-sized sum; the new
//    state is rounded once per step, as in the K scheme.
enum { RK_K = 0, RK_A = 1, RK_D = 2 };
#ifndef SAC_FP32_RK
#define SAC_FP32_RK RK_D
#endif
template <typename T> struct RkScheme { static constexpr int value = SAC_FP32_RK; };
template <> struct RkScheme<double> { static constexpr int value = RK_K; };

template <typename T> __device__ __forceinline__ T tmax(T a, T b) { return fmax(a, b); }
template <> __device__ __forceinline__ float tmax<float>(float a, float b) { return fmaxf(a, b); }
template <typename T> __device__ __forceinline__ T tabs(T a) { return fabs(a); }
template <> __device__ __forceinline__ float tabs<float>(float a) { return fabsf(a); }

__device__ __forceinline__ int wrap_i(int i, int n) { int r = i % n; return r < 0 ? r + n : r; }

// Interior index i plus every ghost index whose boundary rule reads cell i.
__device__ __forceinline__ int ghost_set(int i, int n, int bc, int* list)
{
    int cnt = 0;
    list[cnt++] = i;
    if (bc == BC_PERIODIC) {
        for (int g = -GY; g < 0; ++g) if (wrap_i(g, n) == i) list[cnt++] = g;
        for (int g = n; g < n + GY; ++g) if (wrap_i(g, n) == i) list[cnt++] = g;
    } else if (bc == BC_OUTFLOW) {
        if (i == 0) { list[cnt++] = -1; list[cnt++] = -2; list[cnt++] = -3; }
        if (i == n - 1) { list[cnt++] = n; list[cnt++] = n + 1; list[cnt++] = n + 2; }
    }
    return cnt;
}

template <typename T, int TX, int TY, bool BG>
struct GenericSmem {
    static constexpr int RX = TX + 8, RY = TY + 6, RN = RX * RY;
    static constexpr int NPRIM = 5;   // vx, vy, pt, etot, bv
    static constexpr int NBB = BG ? 2 : 0;
    static constexpr int SN = (TX + 2) * (TY + 2);
    static constexpr int FXN = TY * (TX + 4), FYN = (TY + 4) * TX;
    static constexpr int GXN = TY * (TX + 1), GYN = (TY + 1) * TX;
    static constexpr size_t elems = (size_t)(NF + NBB + NPRIM) * RN + SN + FXN + FYN + GXN + GYN + 64;
    static constexpr size_t bytes = elems * sizeof(T);
};

template <typename T, int STAGE, bool BG, bool HD, int TX, int TY>
__global__ void __launch_bounds__(TX * TY / 2)
stage_generic(const StageArgs<T> a)
{
    using SM = GenericSmem<T, TX, TY, BG>;
    constexpr int RX = SM::RX, RY = SM::RY, RN = SM::RN;
    constexpr int NT = TX * TY / 2;
    constexpr int CPT = 2;                    // cells per thread
    constexpr int VEC = 16 / (int)sizeof(T);  // elements per 16-byte load
    static_assert(RX % VEC == 0, "region width must be a whole number of 16-byte vectors");

    if (a.sc->skip) return;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sU = reinterpret_cast<T*>(smem_raw);              // [NF][RY][RX]
    T* sB = sU + NF * RN;                                // [NBB][RY][RX]  (bbx, bby)
    T* sP = sB + SM::NBB * RN;                           // [5][RY][RX]
    T* sS = sP + SM::NPRIM * RN;                         // [TY+2][TX+2]
    T* sFX = sS + SM::SN;                                // [TY][TX+4]
    T* sFY = sFX + SM::FXN;                              // [TY+4][TX]
    T* sGX = sFY + SM::FYN;                              // [TY][TX+1]
    T* sGY = sGX + SM::GXN;                              // [TY+1][TX]
    __shared__ unsigned long long red[2][NT / 32];

    const Layout L = a.L;
    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    // region (rr, rc) <-> interior (x0 - 4 + rc, y0 - 3 + rr) <-> padded (y0 + rr, x0 + rc)
    const long long rbase = (long long)y0 * L.pitch + x0;

    // ---- stage the stencil input (and background B) -------------------------
    {
        constexpr int VPR = RX / VEC;
        for (int f = 0; f < NF + SM::NBB; ++f) {
            const T* src = (f < NF) ? a.sin + (long long)f * L.fstride
                                    : a.bg + (long long)(2 + f - NF) * L.fstride;
            T* dst = sU + f * RN;
            for (int v = tid; v < RY * VPR; v += NT) {
                int rr = v / VPR, cv = v - rr * VPR;
                const T* g = src + rbase + (long long)rr * L.pitch + cv * VEC;
                if constexpr (sizeof(T) == 4) {
                    float4 q = __ldg(reinterpret_cast<const float4*>(g));
                    *reinterpret_cast<float4*>(dst + rr * RX + cv * VEC) = q;
                } else {
                    double2 q = __ldg(reinterpret_cast<const double2*>(g));
                    *reinterpret_cast<double2*>(dst + rr * RX + cv * VEC) = q;
                }
            }
        }
    }
    __syncthreads();

    const T gm1 = (T)(a.gamma - 1.0);
    const T half = (T)0.5;

    // ---- primitives on the halo box [x0-3, x0+TX+3) x [y0-3, y0+TY+3) -------
    for (int v = tid; v < RY * (RX - 2); v += NT) {
        int rr = v / (RX - 2), rc = 1 + (v - rr * (RX - 2));
        int c = rr * RX + rc;
        T rt = sU[c], mx = sU[RN + c], my = sU[2 * RN + c], et = sU[3 * RN + c];
        T btx = sU[4 * RN + c], bty = sU[5 * RN + c];
        T ux, uy, pt, etot, bv;
        if constexpr (BG) {
            long long gidx = rbase + (long long)rr * L.pitch + rc;
            T rb = __ldg(a.bg + gidx), eb = __ldg(a.bg + L.fstride + gidx);
            T bbx = sB[c], bby = sB[RN + c];
            T rho = rb + rt;
            ux = mx / rho; uy = my / rho;
            T ekin = half * (mx * ux + my * uy);
            T bb = bbx * btx + bby * bty;
            T b2p = half * (btx * btx + bty * bty);
            T pk = gm1 * (((et - ekin) - bb) - b2p);
            pt = (pk + bb) + b2p;
            T b2b = half * (bbx * bbx + bby * bby);
            T pkb = gm1 * (eb - b2b);
            T ptbk = pkb + b2b;
            T bx = bbx + btx, by = bby + bty;
            bv = bx * ux + by * uy;
            etot = ((et + eb) + pt) + ptbk;
        } else {
            T rho = rt;
            ux = mx / rho; uy = my / rho;
            T ekin = half * (mx * ux + my * uy);
            T b2p = half * (btx * btx + bty * bty);
            T pk = gm1 * ((et - ekin) - b2p);
            pt = pk + b2p;
            bv = btx * ux + bty * uy;
            etot = et + pt;
        }
        sP[c] = ux; sP[RN + c] = uy; sP[2 * RN + c] = pt; sP[3 * RN + c] = etot; sP[4 * RN + c] = bv;
    }
    __syncthreads();

    const T d12x = (T)12.0 * (T)a.dx, d12y = (T)12.0 * (T)a.dy;
    const T dxx = (T)a.dx * (T)a.dx, dyy = (T)a.dy * (T)a.dy;

    // ---- shock indicator on [x0-1, x0+TX] x [y0-1, y0+TY] --------------------
    if constexpr (HD) {
        const T* vx = sP;
        const T* vy = sP + RN;
        for (int v = tid; v < SM::SN; v += NT) {
            int sr = v / (TX + 2), scol = v - sr * (TX + 2);
            int c = (sr + 2) * RX + (scol + 3);
            T dvx = ((T)8.0 * (vx[c + 1] - vx[c - 1]) - (vx[c + 2] - vx[c - 2])) / d12x;
            T dvy = ((T)8.0 * (vy[c + RX] - vy[c - RX]) - (vy[c + 2 * RX] - vy[c - 2 * RX])) / d12y;
            T div = dvx + dvy;
            sS[v] = tmax((T)0.0, -div);
        }
    }
    // (the barrier at the top of the variable loop orders sS)

    const T cm[2] = {(T)a.sc->cmax_step[0], (T)a.sc->cmax_step[1]};
    T k[NF][CPT];

#pragma unroll
    for (int f = 0; f < NF; ++f) {
        __syncthreads();   // previous variable's consumers are done with the scratch
        const T* u = sU + f * RN;
        const T* ux = sP; const T* uy = sP + RN; const T* pt = sP + 2 * RN;
        const T* etot = sP + 3 * RN; const T* bv = sP + 4 * RN;
        const T* mx = sU + RN; const T* my = sU + 2 * RN;
        const T* btx = sU + 4 * RN; const T* bty = sU + 5 * RN;
        const T* bbx = sB; const T* bby = sB + RN;

        // x fluxes on cells [x0-2, x0+TX+2) x tile rows
        if (f != 4) {
            for (int v = tid; v < SM::FXN; v += NT) {
                int r = v / (TX + 4), cc = v - r * (TX + 4);
                int c = (r + 3) * RX + (cc + 2);
                T F;
                if (f == 0) F = mx[c];
                else if (f == 1) {
                    if constexpr (BG) F = (ux[c] * mx[c] - ((btx[c] * btx[c] + btx[c] * bbx[c]) + bbx[c] * btx[c])) + pt[c];
                    else F = (ux[c] * mx[c] - btx[c] * btx[c]) + pt[c];
                } else if (f == 2) {
                    if constexpr (BG) F = ux[c] * my[c] - ((btx[c] * bty[c] + btx[c] * bby[c]) + bbx[c] * bty[c]);
                    else F = ux[c] * my[c] - btx[c] * bty[c];
                } else if (f == 3) {
                    T bx = BG ? bbx[c] + btx[c] : btx[c];
                    F = ux[c] * etot[c] - bx * bv[c];
                } else {
                    T bx = BG ? bbx[c] + btx[c] : btx[c];
                    T by = BG ? bby[c] + bty[c] : bty[c];
                    F = ux[c] * by - bx * uy[c];
                }
                sFX[v] = F;
            }
        }
        // y fluxes on tile columns x [y0-2, y0+TY+2)
        if (f != 5) {
            for (int v = tid; v < SM::FYN; v += NT) {
                int r = v / TX, cc = v - r * TX;
                int c = (r + 1) * RX + (cc + 4);
                T F;
                if (f == 0) F = my[c];
                else if (f == 1) {
                    if constexpr (BG) F = uy[c] * mx[c] - ((bty[c] * btx[c] + bty[c] * bbx[c]) + bby[c] * btx[c]);
                    else F = uy[c] * mx[c] - bty[c] * btx[c];
                } else if (f == 2) {
                    if constexpr (BG) F = (uy[c] * my[c] - ((bty[c] * bty[c] + bty[c] * bby[c]) + bby[c] * bty[c])) + pt[c];
                    else F = (uy[c] * my[c] - bty[c] * bty[c]) + pt[c];
                } else if (f == 3) {
                    T by = BG ? bby[c] + bty[c] : bty[c];
                    F = uy[c] * etot[c] - by * bv[c];
                } else {
                    T bx = BG ? bbx[c] + btx[c] : btx[c];
                    T by = BG ? bby[c] + bty[c] : bty[c];
                    F = uy[c] * bx - by * ux[c];
                }
                sFY[v] = F;
            }
        }
        if constexpr (HD) {
            const bool sface = a.hd_single_face != 0;   // ratio from the face itself (variant)
            const T ax = ((T)a.c2[f] * (T)a.dx) * cm[0], ay = ((T)a.c2[f] * (T)a.dy) * cm[1];
            const T bx_ = ((T)a.c_shk * (T)a.dx) * (T)a.dx, by_ = ((T)a.c_shk * (T)a.dy) * (T)a.dy;
            // x faces: face q sits between cells q and q+1, q in [x0-1, x0+TX)
            for (int v = tid; v < SM::GXN; v += NT) {
                int r = v / (TX + 1), q = v - r * (TX + 1);
                int c = (r + 3) * RX + (q + 3);
                T a1[3], a3[3], d1c = (T)0;
#pragma unroll
                for (int o = -1; o <= 1; ++o) {
                    int qq = c + o;
                    T d1 = u[qq + 1] - u[qq];
                    T d3 = (u[qq + 2] - u[qq - 1]) - (T)3.0 * d1;
                    a1[o + 1] = tabs(d1); a3[o + 1] = tabs(d3);
                    if (o == 0) d1c = d1;
                }
                T m1 = sface ? a1[1] : tmax(tmax(a1[0], a1[1]), a1[2]);
                T m3 = sface ? a3[1] : tmax(tmax(a3[0], a3[1]), a3[2]);
                T rr = (m1 > (T)0) ? m3 / m1 : (T)0;
                int sidx = (r + 1) * (TX + 2) + q;   // s at cell q and q+1
                T sf = half * (sS[sidx] + sS[sidx + 1]);
                T nu = ax * rr + bx_ * sf;
                sGX[v] = nu * d1c;
            }
            // y faces: face q between rows q and q+1, q in [y0-1, y0+TY)
            for (int v = tid; v < SM::GYN; v += NT) {
                int q = v / TX, cc = v - q * TX;
                int c = (q + 2) * RX + (cc + 4);
                T a1[3], a3[3], d1c = (T)0;
#pragma unroll
                for (int o = -1; o <= 1; ++o) {
                    int qq = c + o * RX;
                    T d1 = u[qq + RX] - u[qq];
                    T d3 = (u[qq + 2 * RX] - u[qq - RX]) - (T)3.0 * d1;
                    a1[o + 1] = tabs(d1); a3[o + 1] = tabs(d3);
                    if (o == 0) d1c = d1;
                }
                T m1 = sface ? a1[1] : tmax(tmax(a1[0], a1[1]), a1[2]);
                T m3 = sface ? a3[1] : tmax(tmax(a3[0], a3[1]), a3[2]);
                T rr = (m1 > (T)0) ? m3 / m1 : (T)0;
                int sidx = q * (TX + 2) + (cc + 1);
                T sf = half * (sS[sidx] + sS[sidx + TX + 2]);
                T nu = ay * rr + by_ * sf;
                sGY[v] = nu * d1c;
            }
        }
        __syncthreads();
#pragma unroll
        for (int cI = 0; cI < CPT; ++cI) {
            int cx = tid % TX, cy = tid / TX + cI * (TY / CPT);
            T hsum = (T)0;
            if constexpr (HD) {
                T hx = (sGX[cy * (TX + 1) + cx + 1] - sGX[cy * (TX + 1) + cx]) / dxx;
                T hy = (sGY[(cy + 1) * TX + cx] - sGY[cy * TX + cx]) / dyy;
                hsum = hx + hy;
            }
            T dfx = (T)0, dfy = (T)0;
            if (f != 4) {
                const T* F = sFX + cy * (TX + 4) + cx + 2;
                dfx = ((T)8.0 * (F[1] - F[-1]) - (F[2] - F[-2])) / d12x;
            }
            if (f != 5) {
                const T* F = sFY + (cy + 2) * TX + cx;
                dfy = ((T)8.0 * (F[TX] - F[-TX]) - (F[2 * TX] - F[-2 * TX])) / d12y;
            }
            k[f][cI] = hsum - (dfx + dfy);
        }
    }

    // ---- RK update, stage output with ghost copies, signal speed -------------
    const double dtd = a.sc->dt;
    const T dt = (T)dtd, h = (T)(0.5 * dtd), d6 = (T)(dtd / 6.0), d3 = (T)(dtd / 3.0);
    const T third = (T)(1.0 / 3.0);
    const bool edge = (x0 < GY) || (x0 + TX > L.nx - GY) || (y0 < GY) || (y0 + TY > L.ny - GY);
    unsigned long long smax[2] = {0ull, 0ull};
    const bool grav = a.has_grav();
    const T gxv = (T)a.grav[0], gyv = (T)a.grav[1];

#pragma unroll
    for (int cI = 0; cI < CPT; ++cI) {
        int cx = tid % TX, cy = tid / TX + cI * (TY / CPT);
        int i = x0 + cx, j = y0 + cy;
        if (i >= L.nx || j >= L.ny) continue;
        const int c = (cy + 3) * RX + (cx + 4);
        const long long g = L.at(i, j);
        T out[NF];
        // gravity (section 2): rt g in the momentum and m.g in the energy
        // equation, added after the flux and diffusion terms
        T src[NF] = {(T)0, (T)0, (T)0, (T)0, (T)0, (T)0};
        if (grav) {
            const T rt = sU[0 * RN + c], mxc = sU[1 * RN + c], myc = sU[2 * RN + c];
            src[1] = rt * gxv; src[2] = rt * gyv; src[3] = mxc * gxv + myc * gyv;
        }
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            const long long gf = (long long)f * L.fstride + g;
            const T kf = grav && (f >= 1 && f <= 3) ? k[f][cI] + src[f] : k[f][cI];
            constexpr int RK = RkScheme<T>::value;
            if constexpr (RK == RK_K) {
                if (STAGE == 1) {
                    T u0 = sU[f * RN + c];
                    a.acc[gf] = kf;
                    out[f] = u0 + h * kf;
                } else if (STAGE == 2 || STAGE == 3) {
                    T u0 = a.u0[gf];
                    a.acc[gf] = a.acc[gf] + (T)2.0 * kf;
                    out[f] = u0 + (STAGE == 2 ? h : dt) * kf;
                } else {
                    T u0 = a.u0[gf];
                    out[f] = u0 + d6 * (a.acc[gf] + kf);
                }
            } else if constexpr (RK == RK_A) {
                if (STAGE == 1) {
                    out[f] = sU[f * RN + c] + h * kf;
                } else if (STAGE == 2) {
                    T u0 = a.u0[gf];
                    T s1 = sU[f * RN + c];
                    a.acc[gf] = (u0 + third * (s1 - u0)) + d3 * kf;
                    out[f] = u0 + h * kf;
                } else if (STAGE == 3) {
                    T u0 = a.u0[gf];
                    a.acc[gf] = a.acc[gf] + d3 * kf;
                    out[f] = u0 + dt * kf;
                } else {
                    out[f] = a.acc[gf] + d6 * kf;
                }
            } else {
                if (STAGE == 1) {
                    out[f] = sU[f * RN + c] + h * kf;
                } else if (STAGE == 2) {
                    T u0 = a.u0[gf];
                    T s1 = sU[f * RN + c];
                    a.acc[gf] = third * (s1 - u0) + d3 * kf;
                    out[f] = u0 + h * kf;
                } else if (STAGE == 3) {
                    T u0 = a.u0[gf];
                    a.acc[gf] = a.acc[gf] + d3 * kf;
                    out[f] = u0 + dt * kf;
                } else {
                    T u0 = a.u0[gf];
                    out[f] = u0 + (a.acc[gf] + d6 * kf);
                }
            }
        }
        // store (and ghost copies on tiles touching the boundary)
        if (!edge) {
#pragma unroll
            for (int f = 0; f < NF; ++f) a.sout[(long long)f * L.fstride + g] = out[f];
        } else {
            int xs[7], ys[7];
            int nxs = ghost_set(i, L.nx, a.bc_x, xs);
            int nys = ghost_set(j, L.ny, a.bc_y, ys);
            for (int p = 0; p < nys; ++p)
                for (int q = 0; q < nxs; ++q) {
                    long long gg = L.at(xs[q], ys[p]);
#pragma unroll
                    for (int f = 0; f < NF; ++f) a.sout[(long long)f * L.fstride + gg] = out[f];
                }
        }
        if (STAGE == 4) {
            // signal speed of the new state (section 2: sets the next CFL step)
            T sx, sy;
            if constexpr (BG)
                signal_speeds<T, true>(out[0], out[1], out[2], out[3], out[4], out[5],
                                       __ldg(a.bg + g), __ldg(a.bg + L.fstride + g), sB[c], sB[RN + c],
                                       (T)a.gamma, sx, sy);
            else
                signal_speeds<T, false>(out[0], out[1], out[2], out[3], out[4], out[5],
                                        (T)0, (T)0, (T)0, (T)0, (T)a.gamma, sx, sy);
            unsigned long long bxs = speed_key(sx), bys = speed_key(sy);
            smax[0] = bxs > smax[0] ? bxs : smax[0];
            smax[1] = bys > smax[1] ? bys : smax[1];
        }
    }
    if (STAGE == 4) {
#pragma unroll
        for (int d = 0; d < 2; ++d) {
            unsigned long long m = smax[d];
            for (int o = 16; o > 0; o >>= 1) {
                unsigned long long n = __shfl_xor_sync(0xffffffffu, m, o);
                m = n > m ? n : m;
            }
            if ((tid & 31) == 0) red[d][tid >> 5] = m;
        }
        __syncthreads();
        if (tid < 2) {
            unsigned long long m = 0ull;
            for (int w = 0; w < NT / 32; ++w) m = red[tid][w] > m ? red[tid][w] : m;
            atomicMax(&a.sc->cmax_bits[tid], m);
        }
    }
}

}  // namespace sac
