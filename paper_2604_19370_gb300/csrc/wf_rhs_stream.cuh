// Device code of the streaming quadrature (Eq. termsPR tested against every basis function,
// the fuel increment of the Sec. 7 listing and the increment-form right-hand side), shared by
// the per-pass kernels (wf_rhs_stream.cu) and the persistent step kernel (wf_persist.cu).
// The scheme of the computation is described at the top of wf_rhs_stream.cu.
#pragma once
#include <math.h>
#include <stdint.h>

#include <type_traits>

#include "wf_internal.h"

namespace wf {

namespace {

template <typename P>
struct PhysS {
    P K_ign, chiTamb, c_rad, T_amb, T_amb2, C_nld, c_W, T_ig, phi_min, T_a, tau_kf;
    P K0;    // c_chi T_amb + c_rad T_amb^4: the constant part of the point source
    P T_ig_lo;  // T_ig (1 - 1e-5): below it no point of an element row can ignite
    P Ta_l2; // T_a log2(e)
    int heat_by_fuel;
};

// Tables of an interior element (uniform knots: every element p <= e < n - p has the same
// ones), carried in the kernel parameters so that the FMAs read them as constant operands.
template <typename P>
struct ITab {
    P bx[4][4], dx[4][4];  // x: [Gauss point][local basis]
    P by[4][4], dy[4][4];  // y: [Gauss point][local basis]
    P wq[4][4];            // Gauss weight products w_y[b] w_x[q] (every element)
    P wqc[4][4];           // -C_nld w_y[b] w_x[q]
    P wqg[4][4];           // -tau k_f w_y[b] w_x[q]
    // interior y-test tables with the point weights folded in, [b][q][l]:
    P ys[4][4][4];         // B_l(y_b) w_bq               (point source)
    P yd[4][4][4];         // B_l'(y_b) w_bq (-C_nld)     (T^3 dT/dy against dB/dy)
    P yq[4][4][4];         // B_l(y_b) w_bq (-C_nld)      (T^3 dT/dx, tested later against dB/dx)
    P yg[4][4][4];         // B_l(y_b) w_bq (-tau k_f)    (fuel)
    // interior rows of the 1-D mass matrices (rows 2p .. N-1-2p are all equal): the x band
    // A2 = M^x of the second explicit product and the y band B1 = M^y of the first
    P mbx[8], mby[8];
    int xok, yok;          // the interior tables exist (n > 2p)
};

// Tables of the FP32 fast form with the values of Gauss points q = 2j and 2j+1 side by side, so
// that one packed FMA (two FP32 lanes per instruction) serves both points.
struct ITabPairs {
    float2 bx[4][2], dx[4][2];                                  // [k][j]: (B_k(x_2j), B_k(x_2j+1))
    float2 ys[4][4][2], yd[4][4][2], yq[4][4][2], yg[4][4][2];  // [b][l][j], as ITab's y-test tables
};

template <typename P>
struct StreamArgs {
    int nx, ny, Nx, Ny, pitch, seg, nstrips, nsegs;
    int split;  // segments: [0, 2p), interior pieces of [2p, Ny - 2p), [Ny - 2p, Ny)
    int s_lo, s_hi;  // interior strips (every element interior): s_lo <= strip < s_hi
    int seg_b, nseg_b;  // interior segments of the boundary strips: their own height and count
    const P* __restrict__ T;
    const P* __restrict__ phi;
    P* F;
    P* Phi;
    P* R;
    const P *Bx, *Dx, *By, *Dy;
    int wind_rank;
    const P *fxq, *gxq, *fyq, *gyq;
    const P *A1, *B1, *A2, *B2;
    P Rscale, c1, c2;
    PhysS<P> c;
    Batch b;
    ITab<P> it;
    ITabPairs pr;
};

constexpr unsigned FULL = 0xffffffffu;

template <typename P>
__device__ __forceinline__ P col_from(P own, P extra, int lane, int k) {
    // value of the lane `k` to the right; lanes past 31 read the extra column of lane (lane+k-32)
    const P down = __shfl_down_sync(FULL, own, k);
    const P wrap = __shfl_sync(FULL, extra, (lane + k) & 31);
    return (lane + k < 32) ? down : wrap;
}

// exp(-T_a / T).  FP32: 2^(-T_a log2(e) / T) with the fast divide and the hardware base-2
// exponential (PTX ex2.approx, relative error about 2^-22); FP64: exp of the exact quotient.
template <typename P>
__device__ __forceinline__ P arrhenius(const PhysS<P>& c, P T);
template <>
__device__ __forceinline__ float arrhenius<float>(const PhysS<float>& c, float T) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(-__fdividef(c.Ta_l2, T)));
    return y;
}
template <>
__device__ __forceinline__ double arrhenius<double>(const PhysS<double>& c, double T) {
    return exp(-c.T_a / T);
}

// One warp: strip of 32 element columns starting at X0 - p, element rows Y0 - p .. Y1 - 1.
// XI (fast form): every element the warp touches is interior, so all tables come from the
// parameter block; otherwise (boundary strips and the boundary segments) they are read
// through L1.
template <typename P, int PD, int WR, bool XI>
__device__ __forceinline__ void stream_strip(const StreamArgs<P>& a, const ITab<P>& it, int lane, int X0, int Y0,
                                             int Y1) {
    constexpr int Q = PD + 1, NB = PD + 1, W = 2 * PD + 1, NC = 2 * PD + 1;
    const int ex = X0 - PD + lane;             // element column of this lane; also its DOF column
    const bool ex_ok = XI || (ex >= 0 && ex < a.nx);
    const bool out_col = lane >= PD && ex < a.Nx;
    const int cc = ex;                         // coefficient column held by this lane
    const int cc2 = X0 - PD + 32 + lane;       // extra coefficient column (lanes < 2p are used)
    const bool cc_ok = XI || (cc >= 0 && cc < a.Nx);
    const bool cc2_ok = XI || (cc2 >= 0 && cc2 < a.Nx);

    // x tables: interior strips read the parameter block; boundary strips read the element's
    // table through L1 at each use (they are a small share of the work; holding them in
    // registers would raise the register count of every strip)
    const P* __restrict__ Bxe = a.Bx + (size_t)(ex_ok ? ex : 0) * Q * NB;
    const P* __restrict__ Dxe = a.Dx + (size_t)(ex_ok ? ex : 0) * Q * NB;
#define WF_BX(q, k) (XI ? it.bx[q][k] : (ex_ok ? __ldg(Bxe + (q) * NB + (k)) : P(0)))
#define WF_DX(q, k) (XI ? it.dx[q][k] : (ex_ok ? __ldg(Dxe + (q) * NB + (k)) : P(0)))
    // x bands of the DOF column (A1 per scenario; A2 = M^x, from the parameter block on interior
    // strips), and, on interior strips, the y band B2 of the interior DOF rows (per scenario)
    // (the rank-2 wind form keeps the general code here: it has no registers to spare)
    constexpr bool HB2 = XI && WR < 2;
    P a1[W], a2r[W], b2i[W];
#pragma unroll
    for (int d = 0; d < W; ++d) {
        a1[d] = cc_ok ? a.A1[(size_t)cc * W + d] : P(0);
        a2r[d] = (!HB2 && cc_ok && a.A2) ? a.A2[(size_t)cc * W + d] : P(0);
        b2i[d] = (HB2 && a.A2) ? a.B2[(size_t)(2 * PD) * W + d] : P(0);
    }
#define WF_A2(d) (HB2 ? it.mbx[d] : a2r[d])
    P fxr[WR > 0 ? WR : 1][Q], fyr[WR > 0 ? WR : 1][Q];
#pragma unroll
    for (int r = 0; r < WR; ++r)
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            fxr[r][q] = ex_ok ? a.fxq[(size_t)r * a.nx * Q + ex * Q + q] : P(0);
            fyr[r][q] = ex_ok ? a.fyq[(size_t)r * a.nx * Q + ex * Q + q] : P(0);
        }
    // x-test tables of the elements left of this lane: element ex - k, local basis k
    auto tab_left = [&](const P* tab, int k, int q) {
        const int e = ex - k;
        return (e >= 0 && e < a.nx) ? __ldg(tab + ((size_t)e * Q + q) * NB + k) : P(0);
    };
#define WF_TBX(k, q) (XI ? it.bx[q][k] : tab_left(a.Bx, k, q))
#define WF_TDX(k, q) (XI ? it.dx[q][k] : tab_left(a.Dx, k, q))

    // sliding windows
    P xv[NB][Q], xd[NB][Q], xp[NB][Q];  // x-interpolation of coefficient rows ey .. ey+p
    P acs[NB][Q], acq[NB][Q], acg[NB][Q];  // y-test accumulators of DOF rows ey .. ey+p
    P cw1[NC], cw2[NC];                 // x-convolved T rows ey-p .. ey+p (matvec)
#pragma unroll
    for (int l = 0; l < NB; ++l)
#pragma unroll
        for (int q = 0; q < Q; ++q) xv[l][q] = xd[l][q] = xp[l][q] = acs[l][q] = acq[l][q] = acg[l][q] = P(0);
#pragma unroll
    for (int d = 0; d < NC; ++d) cw1[d] = cw2[d] = P(0);

    // coefficient row r: the four values this lane contributes (own and extra column of T and phi)
    struct Row {
        P t0, t1, f0, f1;
    };
    auto fetch_row = [&](int r) {
        Row w;
        const bool rok = r >= 0 && r < a.Ny;
        const size_t o = (size_t)(rok ? r : 0) * a.pitch;
        w.t0 = (rok && cc_ok) ? a.T[o + cc] : P(0);
        w.t1 = (rok && cc2_ok && lane < 2 * PD) ? a.T[o + cc2] : P(0);
        w.f0 = (rok && cc_ok) ? a.phi[o + cc] : P(0);
        w.f1 = (rok && cc2_ok && lane < 2 * PD) ? a.phi[o + cc2] : P(0);
        return w;
    };
    // x-interpolation of a fetched row and its x-convolutions for the matvec
    auto process_row = [&](const Row& w, P(&v)[Q], P(&dv)[Q], P(&pv)[Q], P& w1, P& w2) {
        P ct[NB], cf[NB];
        ct[0] = w.t0;
        cf[0] = w.f0;
#pragma unroll
        for (int k = 1; k < NB; ++k) {
            ct[k] = col_from(w.t0, w.t1, lane, k);
            cf[k] = col_from(w.f0, w.f1, lane, k);
        }
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            P s = 0, sd = 0, sp = 0;
#pragma unroll
            for (int k = 0; k < NB; ++k) {
                s += WF_BX(q, k) * ct[k];
                sd += WF_DX(q, k) * ct[k];
                sp += WF_BX(q, k) * cf[k];
            }
            v[q] = s;
            dv[q] = sd;
            pv[q] = sp;
        }
        P s1 = a1[PD] * w.t0, s2 = WF_A2(PD) * w.t0;
#pragma unroll
        for (int k = 1; k <= PD; ++k) {
            const P up = __shfl_up_sync(FULL, w.t0, k);
            s1 = fma(a1[PD - k], up, fma(a1[PD + k], ct[k], s1));
            s2 = fma(WF_A2(PD - k), up, fma(WF_A2(PD + k), ct[k], s2));
        }
        w1 = s1;
        w2 = s2;
    };

    // one element row: Q x Q points, y-test accumulation into DOF rows ey .. ey+p
    auto element_row = [&](int ey) {
        constexpr bool YI = XI;
        P byr[Q][NB], dyr[Q][NB];
#pragma unroll
        for (int b = 0; b < Q; ++b)
#pragma unroll
            for (int l = 0; l < NB; ++l) {
                byr[b][l] = YI ? P(0) : a.By[(size_t)(ey * Q + b) * NB + l];
                dyr[b][l] = YI ? P(0) : a.Dy[(size_t)(ey * Q + b) * NB + l];
            }
#define WF_BY(b, l) (YI ? it.by[b][l] : byr[b][l])
#define WF_DY(b, l) (YI ? it.dy[b][l] : dyr[b][l])
        P gyr[WR > 0 ? WR : 1][Q], gxr[WR > 0 ? WR : 1][Q];
#pragma unroll
        for (int r = 0; r < WR; ++r)
#pragma unroll
            for (int b = 0; b < Q; ++b) {
                gxr[r][b] = a.gxq[(size_t)r * a.ny * Q + ey * Q + b];
                gyr[r][b] = a.gyq[(size_t)r * a.ny * Q + ey * Q + b];
            }
        const PhysS<P>& c = a.c;
        // no point of the row can reach the ignition temperature unless the largest x-interpolated
        // T of its coefficient rows does (nonnegative y basis values summing to one): one warp
        // vote decides whether the reaction term is evaluated point by point or is zero everywhere
        P m = P(-1e30);
#pragma unroll
        for (int l = 0; l < NB; ++l)
#pragma unroll
            for (int q = 0; q < Q; ++q) m = xv[l][q] > m ? xv[l][q] : m;
        const bool hot = __any_sync(FULL, ex_ok && m > c.T_ig_lo);
        if (!ex_ok) return;
        auto points = [&](auto hot_c) {
        constexpr bool HOT = decltype(hot_c)::value;
#pragma unroll
        for (int b = 0; b < Q; ++b) {
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                P T = 0, Ty = 0, Tx = 0, ph = 0;
#pragma unroll
                for (int l = 0; l < NB; ++l) {
                    T += WF_BY(b, l) * xv[l][q];
                    Ty += WF_DY(b, l) * xv[l][q];
                    Tx += WF_BY(b, l) * xd[l][q];
                    if (HOT) ph += WF_BY(b, l) * xp[l][q];
                }
                P bpx = 0, bpy = 0;
#pragma unroll
                for (int r = 0; r < WR; ++r) {
                    bpx += fxr[r][q] * gxr[r][b];
                    bpy += fyr[r][q] * gyr[r][b];
                }
                // point source: K_ign E (+ c_chi T_amb + c_rad (T_amb^4 - T^4)) - c_W b'.grad T
                const P T2 = T * T, T3 = T2 * T;
                P src = fma(-c.c_rad, T2 * T2, c.K0);
                P EP = P(0);
                if (HOT) {
                    const bool burn = (T > c.T_ig) && (ph > c.phi_min);
                    const P E = burn ? T * arrhenius<P>(c, T) : P(0);
                    EP = E * ph;
                    src = fma(c.K_ign, c.heat_by_fuel ? EP : E, src);
                }
                if (WR > 0) src = fma(-c.c_W, fma(bpx, Tx, bpy * Ty), src);
                const P t3x = T3 * Tx, t3y = T3 * Ty;
                if constexpr (YI) {
#pragma unroll
                    for (int l = 0; l < NB; ++l) {
                        acs[l][q] = fma(it.ys[b][q][l], src, fma(it.yd[b][q][l], t3y, acs[l][q]));
                        acq[l][q] += it.yq[b][q][l] * t3x;
                        if (HOT) acg[l][q] += it.yg[b][q][l] * EP;
                    }
                } else {
                    const P S = it.wq[b][q] * src, QX = it.wqc[b][q] * t3x, QY = it.wqc[b][q] * t3y;
                    const P G = it.wqg[b][q] * EP;
#pragma unroll
                    for (int l = 0; l < NB; ++l) {
                        acs[l][q] = fma(WF_BY(b, l), S, fma(WF_DY(b, l), QY, acs[l][q]));
                        acq[l][q] += WF_BY(b, l) * QX;
                        if (HOT) acg[l][q] += WF_BY(b, l) * G;
                    }
                }
            }
        }
        };
        if (hot)
            points(std::true_type{});
        else
            points(std::false_type{});
#undef WF_BY
#undef WF_DY
    };

    // prologue: rows Y0-2p .. Y0-1 (matvec window), of which Y0-p .. Y0-1 also enter the x window
    const int ey0 = Y0 - PD;
#pragma unroll
    for (int d = 0; d < 2 * PD; ++d) {
        const int r = Y0 - 2 * PD + d;
        P v[Q], dv[Q], pv[Q];
        process_row(fetch_row(r), v, dv, pv, cw1[d], cw2[d]);
        if (d >= PD) {
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                xv[d - PD][q] = v[q];
                xd[d - PD][q] = dv[q];
                xp[d - PD][q] = pv[q];
            }
        }
    }

    Row nxt = fetch_row(ey0 + PD);
    for (int ey = ey0; ey < Y1; ++ey) {
        // new coefficient row ey + p (fetched one iteration ahead), and the fetch of the next one
        const Row cur = nxt;
        nxt = fetch_row(ey + PD + 1);
        process_row(cur, xv[PD], xd[PD], xp[PD], cw1[2 * PD], cw2[2 * PD]);
        if (XI || (ey >= 0 && ey < a.ny)) element_row(ey);
        // DOF row ey is complete: x-test contraction, matvec, stores
        if (ey >= Y0) {
            P Fv = 0, Ph = 0;
#pragma unroll
            for (int k = 0; k < NB; ++k) {
#pragma unroll
                for (int q = 0; q < Q; ++q) {
                    // element ex - k holds DOF column ex as its local basis k
                    const P s = (k == 0) ? acs[0][q] : __shfl_up_sync(FULL, acs[0][q], k);
                    const P u = (k == 0) ? acq[0][q] : __shfl_up_sync(FULL, acq[0][q], k);
                    const P g = (k == 0) ? acg[0][q] : __shfl_up_sync(FULL, acg[0][q], k);
                    Fv = fma(WF_TBX(k, q), s, fma(WF_TDX(k, q), u, Fv));
                    Ph += WF_TBX(k, q) * g;
                }
            }
            if (out_col) {
                const size_t g = (size_t)ey * a.pitch + ex;
                if (a.F) a.F[g] = Fv;
                if (a.Phi) a.Phi[g] = Ph;
                if (a.R) {
                    P r1 = 0, r2 = 0;
                    if constexpr (HB2) {
#pragma unroll
                        for (int d = 0; d < W; ++d) {
                            r1 = fma(it.mby[d], cw1[d], r1);
                            r2 = fma(b2i[d], cw2[d], r2);
                        }
                    } else {
#pragma unroll
                        for (int d = 0; d < W; ++d) {
                            r1 += a.B1[(size_t)ey * W + d] * cw1[d];
                            if (a.A2) r2 += a.B2[(size_t)ey * W + d] * cw2[d];
                        }
                    }
                    a.R[g] = fma(a.Rscale, Fv, fma(a.c1, r1, a.c2 * r2));
                }
            }
        }
        // slide the windows by one row
#pragma unroll
        for (int l = 0; l < PD; ++l)
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                xv[l][q] = xv[l + 1][q];
                xd[l][q] = xd[l + 1][q];
                xp[l][q] = xp[l + 1][q];
                acs[l][q] = acs[l + 1][q];
                acq[l][q] = acq[l + 1][q];
                acg[l][q] = acg[l + 1][q];
            }
#pragma unroll
        for (int q = 0; q < Q; ++q) acs[PD][q] = acq[PD][q] = acg[PD][q] = P(0);
#pragma unroll
        for (int d = 0; d < NC - 1; ++d) {
            cw1[d] = cw1[d + 1];
            cw2[d] = cw2[d + 1];
        }
    }
#undef WF_BX
#undef WF_DX
#undef WF_TBX
#undef WF_TDX
#undef WF_A2
}

// ---- FP32 fast form with packed pairs ---------------------------------------------------
// The computation of stream_strip<float, PD, WR, true> with the Gauss points q = 2j and 2j+1
// of each element row carried side by side in float2 values: interpolation, point source
// and y-test accumulation use packed FMAs (__ffma2_rn: two FP32 FMAs in one instruction),
// which halves the issue slots of that arithmetic; an odd last point stays scalar.  Only
// interior segments take this form, so the y tables are constants; so are the x tables on
// interior strips (XB false), while on the strips that reach the x boundary (XB) each lane
// holds its own element's x tables in registers.
__device__ __forceinline__ float2 f2(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }

template <int PD, int WR, bool XB>
__device__ __forceinline__ void stream_strip_pairs(const StreamArgs<float>& a, const ITab<float>& it,
                                                   const ITabPairs& pt, int lane, int X0, int Y0, int Y1,
                                                   float* wsm) {
    using P = float;
    constexpr int Q = PD + 1, NB = PD + 1, W = 2 * PD + 1, NC = 2 * PD + 1;
    constexpr int QP = Q / 2, QS = Q % 2, QPm = QP > 0 ? QP : 1, WRm = WR > 0 ? WR : 1;
    const int ex = X0 - PD + lane;             // element column of this lane; also its DOF column
    const int cc = ex;                         // coefficient column held by this lane
    const int cc2 = X0 - PD + 32 + lane;       // extra coefficient column (lanes < 2p are used)
    // XB (strips that reach the x boundary): lanes outside [0, nx) carry zero tables, the first
    // and last p element columns their own ones; every lane holds its element's x tables in
    // registers.  Otherwise every element is interior and the tables are constants.
    const bool ex_ok = !XB || (ex >= 0 && ex < a.nx);
    const bool cc_ok = !XB || (cc >= 0 && cc < a.Nx);
    const bool cc2_ok = !XB || (cc2 >= 0 && cc2 < a.Nx);
    const bool out_col = lane >= PD && (!XB || ex < a.Nx);
    float2 rbx[XB ? NB : 1][QPm], rdx[XB ? NB : 1][QPm];
    P rbs[XB ? NB : 1], rds[XB ? NB : 1];
    if constexpr (XB) {
        const P* Be = a.Bx + (size_t)(ex_ok ? ex : 0) * Q * NB;
        const P* De = a.Dx + (size_t)(ex_ok ? ex : 0) * Q * NB;
#pragma unroll
        for (int k = 0; k < NB; ++k) {
#pragma unroll
            for (int j = 0; j < QP; ++j) {
                rbx[k][j] = ex_ok ? make_float2(Be[(2 * j) * NB + k], Be[(2 * j + 1) * NB + k]) : f2(0.f);
                rdx[k][j] = ex_ok ? make_float2(De[(2 * j) * NB + k], De[(2 * j + 1) * NB + k]) : f2(0.f);
            }
            rbs[k] = (QS && ex_ok) ? Be[(Q - 1) * NB + k] : P(0);
            rds[k] = (QS && ex_ok) ? De[(Q - 1) * NB + k] : P(0);
        }
    }
#define WF_PBX(k, j) (XB ? rbx[XB ? k : 0][j] : pt.bx[k][j])
#define WF_PDX(k, j) (XB ? rdx[XB ? k : 0][j] : pt.dx[k][j])
#define WF_SBX(k) (XB ? rbs[XB ? k : 0] : it.bx[Q - 1][k])
#define WF_SDX(k) (XB ? rds[XB ? k : 0] : it.dx[Q - 1][k])
    // x bands of the DOF column: A1 per scenario; A2 = M^x from the constants where every column
    // is interior and the rank-2 wind form needs no registers for it.  Segments of this form are
    // interior in y, so the y band of B2 is its interior row.
    constexpr bool A2C = !XB && WR < 2;
    P a1[W], a2r[W], b2i[W];
#pragma unroll
    for (int d = 0; d < W; ++d) {
        a1[d] = cc_ok ? a.A1[(size_t)cc * W + d] : P(0);
        a2r[d] = (!A2C && cc_ok && a.A2) ? a.A2[(size_t)cc * W + d] : P(0);
        b2i[d] = a.A2 ? a.B2[(size_t)(2 * PD) * W + d] : P(0);
    }
#define WF_A2(d) (A2C ? it.mbx[d] : a2r[d])
    float2 fx2[WRm][QPm], fy2[WRm][QPm];
    P fxs[WRm], fys[WRm];
#pragma unroll
    for (int r = 0; r < WR; ++r) {
        const P* fxp = a.fxq + (size_t)r * a.nx * Q + (size_t)(ex_ok ? ex : 0) * Q;
        const P* fyp = a.fyq + (size_t)r * a.nx * Q + (size_t)(ex_ok ? ex : 0) * Q;
#pragma unroll
        for (int j = 0; j < QP; ++j) {
            fx2[r][j] = ex_ok ? make_float2(fxp[2 * j], fxp[2 * j + 1]) : f2(0.f);
            fy2[r][j] = ex_ok ? make_float2(fyp[2 * j], fyp[2 * j + 1]) : f2(0.f);
        }
        fxs[r] = (QS && ex_ok) ? fxp[Q - 1] : P(0);
        fys[r] = (QS && ex_ok) ? fyp[Q - 1] : P(0);
    }

    // sliding windows: x-interpolated coefficient rows ey .. ey+p, y-test accumulators of DOF rows
    // ey .. ey+p (pairs of Gauss points and the odd last point), x-convolved T rows for the matvec
    float2 xv2[NB][QPm], xd2[NB][QPm], xp2[NB][QPm], as2[NB][QPm], aq2[NB][QPm], ag2[NB][QPm];
    P xvs[NB], xds[NB], xps[NB], ass[NB], aqs[NB], ags[NB];
    P cw1[NC], cw2[NC];
#pragma unroll
    for (int l = 0; l < NB; ++l) {
#pragma unroll
        for (int j = 0; j < QPm; ++j) xv2[l][j] = xd2[l][j] = xp2[l][j] = as2[l][j] = aq2[l][j] = ag2[l][j] = f2(0.f);
        xvs[l] = xds[l] = xps[l] = ass[l] = aqs[l] = ags[l] = P(0);
    }
#pragma unroll
    for (int d = 0; d < NC; ++d) cw1[d] = cw2[d] = P(0);

    struct Row {
        P t0, t1, f0, f1;
    };
    // rows Y0 - 2p .. Y1 + p all exist on an interior segment
    auto fetch_row = [&](int r) {
        Row w;
        const size_t o = (size_t)r * a.pitch;
        w.t0 = cc_ok ? a.T[o + cc] : P(0);
        w.t1 = (cc2_ok && lane < 2 * PD) ? a.T[o + cc2] : P(0);
        w.f0 = cc_ok ? a.phi[o + cc] : P(0);
        w.f1 = (cc2_ok && lane < 2 * PD) ? a.phi[o + cc2] : P(0);
        return w;
    };
    auto process_row = [&](const Row& w, float2(&v)[QPm], float2(&dv)[QPm], float2(&pv)[QPm], P& vs, P& dvs,
                           P& pvs, P& w1, P& w2) {
        P ct[NB], cf[NB];
        ct[0] = w.t0;
        cf[0] = w.f0;
#pragma unroll
        for (int k = 1; k < NB; ++k) {
            ct[k] = col_from(w.t0, w.t1, lane, k);
            cf[k] = col_from(w.f0, w.f1, lane, k);
        }
#pragma unroll
        for (int j = 0; j < QP; ++j) {
            float2 s = mul2(WF_PBX(0, j), f2(ct[0])), sd = mul2(WF_PDX(0, j), f2(ct[0]));
            float2 sp = mul2(WF_PBX(0, j), f2(cf[0]));
#pragma unroll
            for (int k = 1; k < NB; ++k) {
                s = fma2(WF_PBX(k, j), f2(ct[k]), s);
                sd = fma2(WF_PDX(k, j), f2(ct[k]), sd);
                sp = fma2(WF_PBX(k, j), f2(cf[k]), sp);
            }
            v[j] = s;
            dv[j] = sd;
            pv[j] = sp;
        }
        if (QS) {
            P s = 0, sd = 0, sp = 0;
#pragma unroll
            for (int k = 0; k < NB; ++k) {
                s += WF_SBX(k) * ct[k];
                sd += WF_SDX(k) * ct[k];
                sp += WF_SBX(k) * cf[k];
            }
            vs = s;
            dvs = sd;
            pvs = sp;
        }
        P s1 = a1[PD] * w.t0, s2 = WF_A2(PD) * w.t0;
#pragma unroll
        for (int k = 1; k <= PD; ++k) {
            const P up = __shfl_up_sync(FULL, w.t0, k);
            s1 = fma(a1[PD - k], up, fma(a1[PD + k], ct[k], s1));
            s2 = fma(WF_A2(PD - k), up, fma(WF_A2(PD + k), ct[k], s2));
        }
        w1 = s1;
        w2 = s2;
    };

    const PhysS<P>& c = a.c;
    // wind factors of the element rows Y0-p .. Y1-1, staged in this warp's shared memory when the
    // item starts ([r][row][b], x factors then y factors): the rows are then read with short
    // latency, before the row's x interpolation
    const int ey0 = Y0 - PD, nrow = Y1 - ey0;
    if (WR > 0) {
        for (int i = lane; i < WR * nrow * Q; i += 32) {
            const int r = i / (nrow * Q), k = i - r * nrow * Q;
            const size_t g = (size_t)r * a.ny * Q + (size_t)ey0 * Q + k;
            wsm[i] = a.gxq[g];
            wsm[WR * nrow * Q + i] = a.gyq[g];
        }
        __syncwarp();
    }
    P gyr[WRm][Q], gxr[WRm][Q];
    auto load_wind_row = [&](int ey) {
#pragma unroll
        for (int r = 0; r < WR; ++r)
#pragma unroll
            for (int b = 0; b < Q; ++b) {
                gxr[r][b] = wsm[(r * nrow + (ey - ey0)) * Q + b];
                gyr[r][b] = wsm[WR * nrow * Q + (r * nrow + (ey - ey0)) * Q + b];
            }
    };
    // one element row.  HOT: some point may exceed the ignition temperature, so the reaction term
    // is evaluated point by point; otherwise it is zero at every point (E = 0: no reaction source,
    // no fuel change), which is exactly what the point-by-point test would give
    // the odd Gauss point of the x direction at y point b (q = Q - 1, the one-point form)
    auto odd_one = [&](int b, auto hot_c) {
        constexpr bool HOT = decltype(hot_c)::value;
        constexpr int q = Q - 1;
        P T = 0, Ty = 0, Tx = 0, ph = 0;
#pragma unroll
        for (int l = 0; l < NB; ++l) {
            T += it.by[b][l] * xvs[l];
            Ty += it.dy[b][l] * xvs[l];
            Tx += it.by[b][l] * xds[l];
            if (HOT) ph += it.by[b][l] * xps[l];
        }
        P bpx = 0, bpy = 0;
#pragma unroll
        for (int r = 0; r < WR; ++r) {
            bpx += fxs[r] * gxr[r][b];
            bpy += fys[r] * gyr[r][b];
        }
        const P T2 = T * T, T3 = T2 * T;
        P src = fma(-c.c_rad, T2 * T2, c.K0);
        P EP = P(0);
        if (HOT) {
            const bool burn = (T > c.T_ig) && (ph > c.phi_min);
            const P E = burn ? T * arrhenius<P>(c, T) : P(0);
            EP = E * ph;
            src = fma(c.K_ign, c.heat_by_fuel ? EP : E, src);
        }
        if (WR > 0) src = fma(-c.c_W, fma(bpx, Tx, bpy * Ty), src);
        const P t3x = T3 * Tx, t3y = T3 * Ty;
#pragma unroll
        for (int l = 0; l < NB; ++l) {
            ass[l] = fma(it.ys[b][q][l], src, fma(it.yd[b][q][l], t3y, ass[l]));
            aqs[l] = fma(it.yq[b][q][l], t3x, aqs[l]);
            if (HOT) ags[l] = fma(it.yg[b][q][l], EP, ags[l]);
        }
    };
    // the odd Gauss point of the x direction at y points b0 and b0 + 1, side by side in packed FMAs
    // (each lane of a pair computes what odd_one computes for its y point)
    auto odd_pair = [&](int b0, auto hot_c) {
        constexpr bool HOT = decltype(hot_c)::value;
        constexpr int q = Q - 1;
        const int b1 = b0 + 1;
        float2 T = f2(0.f), Ty = f2(0.f), Tx = f2(0.f), ph = f2(0.f);
#pragma unroll
        for (int l = 0; l < NB; ++l) {
            const float2 by = make_float2(it.by[b0][l], it.by[b1][l]), dy = make_float2(it.dy[b0][l], it.dy[b1][l]);
            T = fma2(by, f2(xvs[l]), T);
            Ty = fma2(dy, f2(xvs[l]), Ty);
            Tx = fma2(by, f2(xds[l]), Tx);
            if (HOT) ph = fma2(by, f2(xps[l]), ph);
        }
        float2 bpx = f2(0.f), bpy = f2(0.f);
#pragma unroll
        for (int r = 0; r < WR; ++r) {
            bpx = fma2(f2(fxs[r]), make_float2(gxr[r][b0], gxr[r][b1]), bpx);
            bpy = fma2(f2(fys[r]), make_float2(gyr[r][b0], gyr[r][b1]), bpy);
        }
        const float2 T2 = mul2(T, T), T3 = mul2(T2, T);
        float2 src = fma2(f2(-c.c_rad), mul2(T2, T2), f2(c.K0));
        float2 EP = f2(0.f);
        if (HOT) {
            const bool bx0 = (T.x > c.T_ig) && (ph.x > c.phi_min);
            const bool bx1 = (T.y > c.T_ig) && (ph.y > c.phi_min);
            const float2 E = make_float2(bx0 ? T.x * arrhenius<P>(c, T.x) : P(0),
                                         bx1 ? T.y * arrhenius<P>(c, T.y) : P(0));
            EP = mul2(E, ph);
            src = fma2(f2(c.K_ign), c.heat_by_fuel ? EP : E, src);
        }
        if (WR > 0) src = fma2(f2(-c.c_W), fma2(bpx, Tx, mul2(bpy, Ty)), src);
        const float2 t3x = mul2(T3, Tx), t3y = mul2(T3, Ty);
#pragma unroll
        for (int l = 0; l < NB; ++l) {
            ass[l] = fma(it.ys[b0][q][l], src.x, fma(it.yd[b0][q][l], t3y.x, ass[l]));
            aqs[l] = fma(it.yq[b0][q][l], t3x.x, aqs[l]);
            if (HOT) ags[l] = fma(it.yg[b0][q][l], EP.x, ags[l]);
        }
#pragma unroll
        for (int l = 0; l < NB; ++l) {
            ass[l] = fma(it.ys[b1][q][l], src.y, fma(it.yd[b1][q][l], t3y.y, ass[l]));
            aqs[l] = fma(it.yq[b1][q][l], t3x.y, aqs[l]);
            if (HOT) ags[l] = fma(it.yg[b1][q][l], EP.y, ags[l]);
        }
    };
    auto element_row_body = [&](auto hot_c) {
        constexpr bool HOT = decltype(hot_c)::value;
#pragma unroll
        for (int b = 0; b < Q; ++b) {
#pragma unroll
            for (int j = 0; j < QP; ++j) {
                float2 T = mul2(f2(it.by[b][0]), xv2[0][j]), Ty = mul2(f2(it.dy[b][0]), xv2[0][j]);
                float2 Tx = mul2(f2(it.by[b][0]), xd2[0][j]), ph = f2(0.f);
                if (HOT) ph = mul2(f2(it.by[b][0]), xp2[0][j]);
#pragma unroll
                for (int l = 1; l < NB; ++l) {
                    T = fma2(f2(it.by[b][l]), xv2[l][j], T);
                    Ty = fma2(f2(it.dy[b][l]), xv2[l][j], Ty);
                    Tx = fma2(f2(it.by[b][l]), xd2[l][j], Tx);
                    if (HOT) ph = fma2(f2(it.by[b][l]), xp2[l][j], ph);
                }
                float2 bpx = f2(0.f), bpy = f2(0.f);
#pragma unroll
                for (int r = 0; r < WR; ++r) {
                    bpx = fma2(fx2[r][j], f2(gxr[r][b]), bpx);
                    bpy = fma2(fy2[r][j], f2(gyr[r][b]), bpy);
                }
                const float2 T2 = mul2(T, T);
                const float2 T3 = mul2(T2, T);
                float2 src = fma2(f2(-c.c_rad), mul2(T2, T2), f2(c.K0));
                float2 EP = f2(0.f);
                if (HOT) {
                    const bool bx0 = (T.x > c.T_ig) && (ph.x > c.phi_min);
                    const bool bx1 = (T.y > c.T_ig) && (ph.y > c.phi_min);
                    const float2 E = make_float2(bx0 ? T.x * arrhenius<P>(c, T.x) : P(0),
                                                 bx1 ? T.y * arrhenius<P>(c, T.y) : P(0));
                    EP = mul2(E, ph);
                    src = fma2(f2(c.K_ign), c.heat_by_fuel ? EP : E, src);
                }
                if (WR > 0) src = fma2(f2(-c.c_W), fma2(bpx, Tx, mul2(bpy, Ty)), src);
                const float2 t3x = mul2(T3, Tx), t3y = mul2(T3, Ty);
#pragma unroll
                for (int l = 0; l < NB; ++l) {
                    as2[l][j] = fma2(pt.ys[b][l][j], src, fma2(pt.yd[b][l][j], t3y, as2[l][j]));
                    aq2[l][j] = fma2(pt.yq[b][l][j], t3x, aq2[l][j]);
                    if (HOT) ag2[l][j] = fma2(pt.yg[b][l][j], EP, ag2[l][j]);
                }
            }
        }
        if (QS) {
            // the odd Gauss point of the x direction: y points b and b+1 side by side in packed FMAs,
            // then the last y point alone; per y point the operations, and their order into each
            // accumulator, are those of the one-point form
#pragma unroll
            for (int b = 0; b + 1 < Q; b += 2) odd_pair(b, hot_c);
            if (Q % 2) odd_one(Q - 1, hot_c);
        }
    };

    auto element_row = [&]() {
        // largest x-interpolated T of the element's coefficient rows: the y interpolation, with
        // nonnegative basis values summing to one, cannot exceed it at any point
        P m = QS ? xvs[0] : xv2[0][0].x;
#pragma unroll
        for (int l = 0; l < NB; ++l) {
#pragma unroll
            for (int j = 0; j < QP; ++j) m = fmaxf(m, fmaxf(xv2[l][j].x, xv2[l][j].y));
            if (QS) m = fmaxf(m, xvs[l]);
        }
        if (__any_sync(FULL, m > c.T_ig_lo))
            element_row_body(std::true_type{});
        else
            element_row_body(std::false_type{});
    };

    // prologue: rows Y0-2p .. Y0-1 (matvec window), of which Y0-p .. Y0-1 also enter the x window
#pragma unroll
    for (int d = 0; d < 2 * PD; ++d) {
        const int r = Y0 - 2 * PD + d;
        float2 v[QPm], dv[QPm], pv[QPm];
        P vs = 0, dvs = 0, pvs = 0;
        process_row(fetch_row(r), v, dv, pv, vs, dvs, pvs, cw1[d], cw2[d]);
        if (d >= PD) {
#pragma unroll
            for (int j = 0; j < QP; ++j) {
                xv2[d - PD][j] = v[j];
                xd2[d - PD][j] = dv[j];
                xp2[d - PD][j] = pv[j];
            }
            xvs[d - PD] = vs;
            xds[d - PD] = dvs;
            xps[d - PD] = pvs;
        }
    }

    Row nxt = fetch_row(ey0 + PD);
    for (int ey = ey0; ey < Y1; ++ey) {
        const Row cur = nxt;
        nxt = fetch_row(ey + PD + 1);
        load_wind_row(ey);
        process_row(cur, xv2[PD], xd2[PD], xp2[PD], xvs[PD], xds[PD], xps[PD], cw1[2 * PD], cw2[2 * PD]);
        element_row();
        if (ey >= Y0) {
            // x-test contraction: each lane first folds its own element's contributions to its
            // local basis functions k (with its own x tables), then DOF column ex gathers local
            // basis k of element ex - k from the lane k to its left
            P Fv = 0, Ph = 0;
#pragma unroll
            for (int k = 0; k < NB; ++k) {
                float2 C2 = mul2(WF_PDX(k, 0), aq2[0][0]);
                C2 = fma2(WF_PBX(k, 0), as2[0][0], C2);
                float2 G2 = mul2(WF_PBX(k, 0), ag2[0][0]);
#pragma unroll
                for (int j = 1; j < QP; ++j) {
                    C2 = fma2(WF_PBX(k, j), as2[0][j], fma2(WF_PDX(k, j), aq2[0][j], C2));
                    G2 = fma2(WF_PBX(k, j), ag2[0][j], G2);
                }
                P Ck = C2.x + C2.y, Gk = G2.x + G2.y;
                if (QS) {
                    Ck = fma(WF_SBX(k), ass[0], fma(WF_SDX(k), aqs[0], Ck));
                    Gk = fma(WF_SBX(k), ags[0], Gk);
                }
                if (k > 0) {
                    Ck = __shfl_up_sync(FULL, Ck, k);
                    Gk = __shfl_up_sync(FULL, Gk, k);
                }
                Fv += Ck;
                Ph += Gk;
            }
            if (out_col) {
                const size_t g = (size_t)ey * a.pitch + ex;
                if (a.F) a.F[g] = Fv;
                if (a.Phi) a.Phi[g] = Ph;
                if (a.R) {
                    P r1 = 0, r2 = 0;
#pragma unroll
                    for (int d = 0; d < W; ++d) {
                        r1 = fma(it.mby[d], cw1[d], r1);
                        r2 = fma(b2i[d], cw2[d], r2);
                    }
                    a.R[g] = fma(a.Rscale, Fv, fma(a.c1, r1, a.c2 * r2));
                }
            }
        }
        // slide the windows by one row
#pragma unroll
        for (int l = 0; l < PD; ++l) {
#pragma unroll
            for (int j = 0; j < QPm; ++j) {
                xv2[l][j] = xv2[l + 1][j];
                xd2[l][j] = xd2[l + 1][j];
                xp2[l][j] = xp2[l + 1][j];
                as2[l][j] = as2[l + 1][j];
                aq2[l][j] = aq2[l + 1][j];
                ag2[l][j] = ag2[l + 1][j];
            }
            xvs[l] = xvs[l + 1];
            xds[l] = xds[l + 1];
            xps[l] = xps[l + 1];
            ass[l] = ass[l + 1];
            aqs[l] = aqs[l + 1];
            ags[l] = ags[l + 1];
        }
#pragma unroll
        for (int j = 0; j < QPm; ++j) as2[PD][j] = aq2[PD][j] = ag2[PD][j] = f2(0.f);
        ass[PD] = aqs[PD] = ags[PD] = P(0);
#pragma unroll
        for (int d = 0; d < NC - 1; ++d) {
            cw1[d] = cw1[d + 1];
            cw2[d] = cw2[d + 1];
        }
    }
#undef WF_A2
#undef WF_PBX
#undef WF_PDX
#undef WF_SBX
#undef WF_SDX
}

template <typename P>
PhysS<P> to_phys_s(const Phys& c, double tau) {
    PhysS<P> o;
    o.K_ign = (P)c.K_ign;
    o.chiTamb = (P)(c.c_chi * c.T_amb);
    o.c_rad = (P)c.c_rad;
    o.T_amb = (P)c.T_amb;
    o.T_amb2 = (P)(c.T_amb * c.T_amb);
    o.C_nld = (P)c.C_nld;
    o.c_W = (P)c.c_W;
    o.T_ig = (P)c.T_ig;
    o.T_ig_lo = (P)(c.T_ig * (1.0 - 1e-5));
    o.phi_min = (P)c.phi_min;
    o.T_a = (P)c.T_a;
    o.tau_kf = (P)(tau * c.k_f);
    o.K0 = (P)(c.c_chi * c.T_amb + c.c_rad * c.T_amb * c.T_amb * c.T_amb * c.T_amb);
    o.Ta_l2 = (P)(c.T_a * 1.4426950408889634074);  // log2(e)
    o.heat_by_fuel = c.heat_by_fuel;
    return o;
}

// Kernel arguments of the streaming quadrature for segments of `seg` element rows (everything
// but the boundary-strip segments of the split launches, seg_b / nseg_b, which stay zero).
template <typename P, int PD>
void fill_stream_args(const RhsArgs& r, int seg, StreamArgs<P>& a) {
    a.nx = r.nx;
    a.ny = r.ny;
    a.Nx = r.Nx;
    a.Ny = r.Ny;
    a.pitch = r.pitch;
    a.nstrips = (r.Nx + (32 - PD) - 1) / (32 - PD);
    a.seg = seg;
    a.seg_b = a.nseg_b = 0;
    a.T = (const P*)r.T;
    a.phi = (const P*)r.phi;
    a.F = (P*)r.F;
    a.Phi = (P*)r.Phi;
    a.R = (P*)r.R;
    a.Bx = (const P*)r.Bx;
    a.Dx = (const P*)r.Dx;
    a.By = (const P*)r.By;
    a.Dy = (const P*)r.Dy;
    a.wind_rank = r.wind_rank;
    a.fxq = (const P*)r.fxq;
    a.gxq = (const P*)r.gxq;
    a.fyq = (const P*)r.fyq;
    a.gyq = (const P*)r.gyq;
    a.A1 = (const P*)r.A1;
    a.B1 = (const P*)r.B1;
    a.A2 = (const P*)r.A2;
    a.B2 = (const P*)r.B2;
    a.Rscale = (P)r.Rscale;
    a.c1 = (P)r.c1;
    a.c2 = (P)r.c2;
    a.c = to_phys_s<P>(r.phys, r.tau);
    a.b = r.b;
    // interior segments need element rows p .. ny-p-1 only: the middle [2p, Ny - 2p) is cut
    // into pieces, the 2p DOF rows at either end form their own (boundary) segments
    const int mid = r.Ny - 4 * PD;
    a.split = (r.tx.ok && r.ty.ok && mid >= 1) ? 1 : 0;
    a.nsegs = a.split ? 2 + (mid + seg - 1) / seg : (r.Ny + seg - 1) / seg;
    // interior strips: X0 = s (32 - p) >= 2p and X0 + 31 < nx (a contiguous range of s)
    a.s_lo = a.s_hi = 0;
    if (r.tx.ok) {
        int lo = -1, hi = -1;
        for (int st = 0; st < a.nstrips; ++st) {
            const int X0 = st * (32 - PD);
            if (X0 >= 2 * PD && X0 + 31 < r.nx) {
                if (lo < 0) lo = st;
                hi = st + 1;
            }
        }
        if (lo >= 0) {
            a.s_lo = lo;
            a.s_hi = hi;
        }
    }
    for (int i = 0; i < 4; ++i) {
        for (int j = 0; j < 4; ++j) {
            a.it.bx[i][j] = (P)r.tx.B[i][j];
            a.it.dx[i][j] = (P)r.tx.D[i][j];
            a.it.by[i][j] = (P)r.ty.B[i][j];
            a.it.dy[i][j] = (P)r.ty.D[i][j];
        }
        for (int j = 0; j < 4; ++j) {
            const double wq = r.ty.w[i] * r.tx.w[j];
            a.it.wq[i][j] = (P)wq;
            a.it.wqc[i][j] = (P)(-wq * r.phys.C_nld);
            a.it.wqg[i][j] = (P)(-wq * r.tau * r.phys.k_f);
            for (int l = 0; l < 4; ++l) {
                a.it.ys[i][j][l] = (P)(r.ty.B[i][l] * wq);
                a.it.yd[i][j][l] = (P)(r.ty.D[i][l] * wq * -r.phys.C_nld);
                a.it.yq[i][j][l] = (P)(r.ty.B[i][l] * wq * -r.phys.C_nld);
                a.it.yg[i][j][l] = (P)(r.ty.B[i][l] * wq * -(r.tau * r.phys.k_f));
            }
        }
    }
    for (int k = 0; k < 4; ++k)
        for (int j = 0; j < 2; ++j) {
            const int q0 = 2 * j, q1 = 2 * j + 1;
            a.pr.bx[k][j] = make_float2((float)r.tx.B[q0][k], (float)r.tx.B[q1][k]);
            a.pr.dx[k][j] = make_float2((float)r.tx.D[q0][k], (float)r.tx.D[q1][k]);
            for (int b = 0; b < 4; ++b) {
                const double w0 = r.ty.w[b] * r.tx.w[q0], w1 = r.ty.w[b] * r.tx.w[q1];
                const double Bb = r.ty.B[b][k], Db = r.ty.D[b][k];
                const double cn = -r.phys.C_nld, cg = -(r.tau * r.phys.k_f);
                a.pr.ys[b][k][j] = make_float2((float)(Bb * w0), (float)(Bb * w1));
                a.pr.yd[b][k][j] = make_float2((float)(Db * w0 * cn), (float)(Db * w1 * cn));
                a.pr.yq[b][k][j] = make_float2((float)(Bb * w0 * cn), (float)(Bb * w1 * cn));
                a.pr.yg[b][k][j] = make_float2((float)(Bb * w0 * cg), (float)(Bb * w1 * cg));
            }
        }
    for (int d = 0; d < 8; ++d) {
        a.it.mbx[d] = (P)r.tx.Mb[d];
        a.it.mby[d] = (P)r.ty.Mb[d];
    }
    a.it.xok = r.tx.ok;
    a.it.yok = r.ty.ok;
}

}  // namespace
}  // namespace wf
