// Explicit right-hand side by sum-factorised Gauss quadrature.
//
// Paper: the nonlinear terms F of Eq. termsPR (normalised form at the start of
// Sec. 3) tested against every basis function, and the fuel load vector of the
// explicit Euler update in the right-hand-side listing of Sec. 7:
//
//   F_ij   = sum_e sum_pts W [ s B_i B_j - c_W (b'.grad T) B_i B_j
//                              + q (T_x B_i' B_j + T_y B_i B_j') ]
//   Phi_ij = sum_e sum_pts W (-tau k_f E phi) B_i B_j    (increment form of the fuel update:
//            int phi B_i B_j = ((M (x) M) phi)_ij exactly, so phi^{n+1} = phi + (M (x) M)^{-1} Phi)
//   s = K_ign E + c_chi T_amb + c_rad (T_amb^4 - T^4),  E = [T > T_ig, phi > phi_min] T e^{-T_a/T},
//   q = -C_nld T^3
//
// and, in the same pass, the right-hand side of the scheme in increment form,
//   R = Rscale F + c1 (A1^x (x) B1^y) T + c2 (A2^x (x) B2^y) T,
// e.g. for the first PR substep R = (tau/2) F - (tau/2)(A_x (x) M^y) T - (tau/2)(M^x (x) A_y) T,
// whose solution is the increment T* - T (the same system as Eq. matrixPR with the
// identity (M^x (x) Y_-) T = (X_+ (x) M^y) T - (tau/2)(A_x (x) M + M (x) A_y) T moved to the left).
//
// One CTA computes a TJ x TI tile of output coefficients.  It stages the
// (TJ+2p) x (TI+2p) halo of T and phi in shared memory and evaluates the
// elements touching the tile by sum factorisation: contraction along x to the
// x Gauss points, then along y to the points, the pointwise terms, the test
// contraction along y and finally along x.  Elements on the tile border are
// evaluated by both neighbouring tiles (gather form: no atomics, results are
// bitwise reproducible).
#include <math.h>

#include "wf_internal.h"

namespace wf {

namespace {

template <typename P>
struct PhysP {
    P K_ign, chiTamb, c_rad, T_amb, T_amb2, C_nld, c_W, T_ig, phi_min, T_a, tau_kf;
    int heat_by_fuel;
};

template <typename P>
__device__ __forceinline__ P expo(P x);
template <>
__device__ __forceinline__ float expo<float>(float x) { return __expf(x); }
template <>
__device__ __forceinline__ double expo<double>(double x) { return exp(x); }

template <typename P>
__device__ __forceinline__ void pointwise(P T, P Tx, P Ty, P phi, P bpx, P bpy, P W, const PhysP<P>& c, P& S, P& QX,
                                          P& QY, P& G) {
    const bool burn = (T > c.T_ig) && (phi > c.phi_min);
    const P E = burn ? T * expo<P>(-c.T_a / T) : P(0);
    const P T2 = T * T;
    // c_rad (T_amb^4 - T^4) in factored form: exact zero at T = T_amb
    const P rad = c.c_rad * (c.T_amb2 + T2) * (c.T_amb + T) * (c.T_amb - T);
    const P heat = c.K_ign * E * (c.heat_by_fuel ? phi : P(1));
    const P s = heat + c.chiTamb + rad - c.c_W * (bpx * Tx + bpy * Ty);
    const P q = -c.C_nld * T2 * T;
    S = W * s;
    QX = W * q * Tx;
    QY = W * q * Ty;
    G = -W * c.tau_kf * E * phi;
}

template <typename P>
struct RhsArgsT {
    int nx, ny, Nx, Ny, pitch;
    const P* __restrict__ T;
    const P* __restrict__ phi;
    P* F;
    P* Phi;
    P* R;
    const P *Bx, *Dx, *By, *Dy, *wx, *wy;
    int wind_rank;
    const P *fxq, *gxq, *fyq, *gyq;
    const P *A1, *B1, *A2, *B2;
    P Rscale, c1, c2;
    PhysP<P> c;
    Batch b;
};

template <typename P, int PD, int TJ, int TI>
struct RhsShape {
    static constexpr int Q = PD + 1, NB = PD + 1;
    static constexpr int CJ = TJ + 2 * PD, CI = TI + 2 * PD;  // coefficient halo tile
    static constexpr int EJ = TJ + PD, EI = TI + PD;          // elements touching the tile
    static constexpr int XI = EI * Q, YJ = EJ * Q;            // Gauss points of those elements
    static constexpr int nP = 2 * CJ * CI + 3 * CJ * XI + 4 * YJ * XI + 3 * TJ * XI;
    static constexpr size_t bytes = sizeof(P) * nP;
};

template <typename P, int PD, int TJ, int TI, int NT>
__global__ void __launch_bounds__(NT) k_rhs(const RhsArgsT<P> a_in) {
    using S_ = RhsShape<P, PD, TJ, TI>;
    if (!scene_active(a_in.b)) return;
    RhsArgsT<P> a = a_in;
    a.T = scene_ptr(a.T, a.b);
    a.phi = scene_ptr(a.phi, a.b);
    a.F = scene_ptr(a.F, a.b);
    a.Phi = scene_ptr(a.Phi, a.b);
    a.R = scene_ptr(a.R, a.b);
    a.A1 = scene_ptr(a.A1, a.b);
    a.B1 = scene_ptr(a.B1, a.b);
    a.A2 = scene_ptr(a.A2, a.b);
    a.B2 = scene_ptr(a.B2, a.b);
    a.fxq = scene_ptr(a.fxq, a.b);
    a.gxq = scene_ptr(a.gxq, a.b);
    a.fyq = scene_ptr(a.fyq, a.b);
    a.gyq = scene_ptr(a.gyq, a.b);
    constexpr int Q = S_::Q, NB = S_::NB, CJ = S_::CJ, CI = S_::CI, EJ = S_::EJ, EI = S_::EI, XI = S_::XI,
                  YJ = S_::YJ;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    P* cT = reinterpret_cast<P*>(smem_raw);
    P* cP = cT + CJ * CI;
    P* xv = cP + CJ * CI;
    P* xd = xv + CJ * XI;
    P* xp = xd + CJ * XI;
    P* pS = xp + CJ * XI;
    P* pQX = pS + YJ * XI;
    P* pQY = pQX + YJ * XI;
    P* pG = pQY + YJ * XI;
    P* ys = pG + YJ * XI;
    P* yq = ys + TJ * XI;
    P* yg = yq + TJ * XI;

    const int i0 = blockIdx.x * TI, j0 = blockIdx.y * TJ;
    const int tid = threadIdx.x;

    // A: halo of coefficients (zero outside the domain)
    for (int idx = tid; idx < CJ * CI; idx += NT) {
        const int cy = idx / CI, cx = idx - cy * CI;
        const int gj = j0 - PD + cy, gi = i0 - PD + cx;
        const bool ok = gj >= 0 && gj < a.Ny && gi >= 0 && gi < a.Nx;
        const size_t g = (size_t)gj * a.pitch + gi;
        cT[idx] = ok ? a.T[g] : P(0);
        cP[idx] = ok ? a.phi[g] : P(0);
    }
    __syncthreads();

    // B: contraction along x: coefficient row cy, element lx -> its Q x-points
    for (int idx = tid; idx < CJ * EI; idx += NT) {
        const int cy = idx / EI, lx = idx - cy * EI;
        const int ex = i0 - PD + lx;
        P c[NB], f[NB];
#pragma unroll
        for (int k = 0; k < NB; ++k) {
            c[k] = cT[cy * CI + lx + k];
            f[k] = cP[cy * CI + lx + k];
        }
        const bool ok = ex >= 0 && ex < a.nx;
#pragma unroll
        for (int aq = 0; aq < Q; ++aq) {
            P v = 0, d = 0, fp = 0;
            if (ok) {
                const P* Bt = a.Bx + (size_t)(ex * Q + aq) * NB;
                const P* Dt = a.Dx + (size_t)(ex * Q + aq) * NB;
#pragma unroll
                for (int k = 0; k < NB; ++k) {
                    v += Bt[k] * c[k];
                    d += Dt[k] * c[k];
                    fp += Bt[k] * f[k];
                }
            }
            xv[cy * XI + lx * Q + aq] = v;
            xd[cy * XI + lx * Q + aq] = d;
            xp[cy * XI + lx * Q + aq] = fp;
        }
    }
    __syncthreads();

    // C: contraction along y to the points, then the pointwise terms
    for (int idx = tid; idx < EJ * XI; idx += NT) {
        const int ly = idx / XI, px = idx - ly * XI;
        const int lx = px / Q, aq = px - lx * Q;
        const int ey = j0 - PD + ly, ex = i0 - PD + lx;
        const bool ok = ey >= 0 && ey < a.ny && ex >= 0 && ex < a.nx;
        P cv[NB], cd[NB], cf[NB];
#pragma unroll
        for (int l = 0; l < NB; ++l) {
            cv[l] = xv[(ly + l) * XI + px];
            cd[l] = xd[(ly + l) * XI + px];
            cf[l] = xp[(ly + l) * XI + px];
        }
#pragma unroll
        for (int b = 0; b < Q; ++b) {
            P S = 0, QX = 0, QY = 0, G = 0;
            if (ok) {
                const P* Bt = a.By + (size_t)(ey * Q + b) * NB;
                const P* Dt = a.Dy + (size_t)(ey * Q + b) * NB;
                P T = 0, Ty = 0, Tx = 0, ph = 0;
#pragma unroll
                for (int l = 0; l < NB; ++l) {
                    T += Bt[l] * cv[l];
                    Ty += Dt[l] * cv[l];
                    Tx += Bt[l] * cd[l];
                    ph += Bt[l] * cf[l];
                }
                P bpx = 0, bpy = 0;
                for (int r = 0; r < a.wind_rank; ++r) {
                    bpx += a.fxq[(size_t)r * a.nx * Q + ex * Q + aq] * a.gxq[(size_t)r * a.ny * Q + ey * Q + b];
                    bpy += a.fyq[(size_t)r * a.nx * Q + ex * Q + aq] * a.gyq[(size_t)r * a.ny * Q + ey * Q + b];
                }
                pointwise<P>(T, Tx, Ty, ph, bpx, bpy, a.wx[aq] * a.wy[b], a.c, S, QX, QY, G);
            }
            const int py = ly * Q + b;
            pS[py * XI + px] = S;
            pQX[py * XI + px] = QX;
            pQY[py * XI + px] = QY;
            pG[py * XI + px] = G;
        }
    }
    __syncthreads();

    // D: test contraction along y: output row jl, x-point px
    for (int idx = tid; idx < TJ * XI; idx += NT) {
        const int jl = idx / XI, px = idx - jl * XI;
        const int j = j0 + jl;
        P s = 0, qq = 0, g = 0;
#pragma unroll
        for (int l = 0; l < NB; ++l) {
            const int ey = j - l;
            if (ey < 0 || ey >= a.ny) continue;
            const int ly = jl + PD - l;
#pragma unroll
            for (int b = 0; b < Q; ++b) {
                const P Bt = a.By[(size_t)(ey * Q + b) * NB + l];
                const P Dt = a.Dy[(size_t)(ey * Q + b) * NB + l];
                const int o = (ly * Q + b) * XI + px;
                s += Bt * pS[o] + Dt * pQY[o];
                qq += Bt * pQX[o];
                g += Bt * pG[o];
            }
        }
        ys[jl * XI + px] = s;
        yq[jl * XI + px] = qq;
        yg[jl * XI + px] = g;
    }
    __syncthreads();

    // E: test contraction along x, Kronecker matvec, stores
    for (int idx = tid; idx < TJ * TI; idx += NT) {
        const int jl = idx / TI, il = idx - jl * TI;
        const int i = i0 + il, j = j0 + jl;
        if (i >= a.Nx || j >= a.Ny) continue;
        P Fv = 0, Ph = 0;
#pragma unroll
        for (int k = 0; k < NB; ++k) {
            const int ex = i - k;
            if (ex < 0 || ex >= a.nx) continue;
            const int lx = il + PD - k;
#pragma unroll
            for (int aq = 0; aq < Q; ++aq) {
                const P Bt = a.Bx[(size_t)(ex * Q + aq) * NB + k];
                const P Dt = a.Dx[(size_t)(ex * Q + aq) * NB + k];
                const int o = jl * XI + lx * Q + aq;
                Fv += Bt * ys[o] + Dt * yq[o];
                Ph += Bt * yg[o];
            }
        }
        const size_t g = (size_t)j * a.pitch + i;
        if (a.F) a.F[g] = Fv;
        if (a.Phi) a.Phi[g] = Ph;
        if (a.R) {
            constexpr int W = 2 * PD + 1;
            P r1 = 0, r2 = 0;
#pragma unroll
            for (int dl = 0; dl < W; ++dl) {
                P t = 0;
#pragma unroll
                for (int dk = 0; dk < W; ++dk) t += a.A1[(size_t)i * W + dk] * cT[(jl + dl) * CI + il + dk];
                r1 += a.B1[(size_t)j * W + dl] * t;
            }
            if (a.A2) {
#pragma unroll
                for (int dl = 0; dl < W; ++dl) {
                    P t = 0;
#pragma unroll
                    for (int dk = 0; dk < W; ++dk) t += a.A2[(size_t)i * W + dk] * cT[(jl + dl) * CI + il + dk];
                    r2 += a.B2[(size_t)j * W + dl] * t;
                }
            }
            a.R[g] = a.Rscale * Fv + a.c1 * r1 + a.c2 * r2;
        }
    }
}

template <typename P>
PhysP<P> to_phys(const Phys& c, double tau) {
    PhysP<P> o;
    o.K_ign = (P)c.K_ign;
    o.chiTamb = (P)(c.c_chi * c.T_amb);
    o.c_rad = (P)c.c_rad;
    o.T_amb = (P)c.T_amb;
    o.T_amb2 = (P)(c.T_amb * c.T_amb);
    o.C_nld = (P)c.C_nld;
    o.c_W = (P)c.c_W;
    o.T_ig = (P)c.T_ig;
    o.phi_min = (P)c.phi_min;
    o.T_a = (P)c.T_a;
    o.tau_kf = (P)(tau * c.k_f);
    o.heat_by_fuel = c.heat_by_fuel;
    return o;
}

template <typename P>
RhsArgsT<P> to_typed(const RhsArgs& a) {
    RhsArgsT<P> t;
    t.nx = a.nx;
    t.ny = a.ny;
    t.Nx = a.Nx;
    t.Ny = a.Ny;
    t.pitch = a.pitch;
    t.T = (const P*)a.T;
    t.phi = (const P*)a.phi;
    t.F = (P*)a.F;
    t.Phi = (P*)a.Phi;
    t.R = (P*)a.R;
    t.Bx = (const P*)a.Bx;
    t.Dx = (const P*)a.Dx;
    t.By = (const P*)a.By;
    t.Dy = (const P*)a.Dy;
    t.wx = (const P*)a.wx;
    t.wy = (const P*)a.wy;
    t.wind_rank = a.wind_rank;
    t.fxq = (const P*)a.fxq;
    t.gxq = (const P*)a.gxq;
    t.fyq = (const P*)a.fyq;
    t.gyq = (const P*)a.gyq;
    t.A1 = (const P*)a.A1;
    t.B1 = (const P*)a.B1;
    t.A2 = (const P*)a.A2;
    t.B2 = (const P*)a.B2;
    t.Rscale = (P)a.Rscale;
    t.c1 = (P)a.c1;
    t.c2 = (P)a.c2;
    t.c = to_phys<P>(a.phys, a.tau);
    t.b = a.b;
    return t;
}

template <typename P, int PD, int TJ, int TI, int NT>
cudaError_t run_rhs(const RhsArgs& a, cudaStream_t s) {
    using S_ = RhsShape<P, PD, TJ, TI>;
    auto kern = k_rhs<P, PD, TJ, TI, NT>;
    static bool configured = false;
    if (!configured) {
        cudaError_t e = allow_dynamic_smem(kern, (size_t)S_::bytes);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    dim3 grid((a.Nx + TI - 1) / TI, (a.Ny + TJ - 1) / TJ, a.b.S);
    kern<<<grid, NT, S_::bytes, s>>>(to_typed<P>(a));
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_rhs(int prec, int p, const RhsArgs& a, cudaStream_t s) {
    cudaError_t e = launch_rhs_stream(prec, p, a, s);
    if (e != cudaErrorNotSupported) return e;
    cudaGetLastError();
    return launch_rhs_tile(prec, p, a, s);
}

cudaError_t launch_rhs_tile(int prec, int p, const RhsArgs& a, cudaStream_t s) {
    if (prec == 0) {
        switch (p) {
            case 1: return run_rhs<float, 1, 16, 16, 256>(a, s);
            case 2: return run_rhs<float, 2, 16, 16, 256>(a, s);
            case 3: return run_rhs<float, 3, 16, 16, 256>(a, s);
        }
    } else {
        switch (p) {
            case 1: return run_rhs<double, 1, 16, 16, 256>(a, s);
            case 2: return run_rhs<double, 2, 16, 16, 256>(a, s);
            case 3: return run_rhs<double, 3, 8, 8, 128>(a, s);
        }
    }
    return cudaErrorInvalidValue;
}

int rhs_items_per_dof(int p) { return (p + 1) * (p + 1); }

}  // namespace wf
