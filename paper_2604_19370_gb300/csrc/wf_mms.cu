// Manufactured-solution forcing of the convergence study (Sec. 6, "Stability and order of the
// time integration scheme").
//
// The exact solution is u*(x, y, t) = base + sum_k A_k (1 - cos(2 pi n_k x / L_x))
// (1 - cos(2 pi m_k y / L_y)) exp(-lambda_k t); the forcing that makes it solve the model is
//   f = u_t - C_d lap u + c_W b.grad u + c_chi u
//       - [c_chi T_amb + c_rad (T_amb^4 - u^4) + C_nld (u^3 lap u + 3 u^2 |grad u|^2)]
// at u* (combustion and wind variation off in the study).  k_forcing adds
// s1 * int f(., t) B_i B_j to one array and s2 * the same to another, by the q-point Gauss
// rule of the load vectors, t read from device memory so that captured graphs stay valid;
// k_advance_time moves t by one step.  Everything here runs in FP64.
#include <math.h>

#include "wf_internal.h"

namespace wf {

namespace {

__device__ double mms_forcing(const MmsArgs& a, double x, double y, double t) {
    double u = a.base, ut = 0, ux = 0, uy = 0, uxx = 0, uyy = 0;
    for (int k = 0; k < a.nmodes; ++k) {
        const double kx = 2.0 * M_PI * a.kx[k] / a.Lx, ky = 2.0 * M_PI * a.ky[k] / a.Ly;
        const double e = a.amp[k] * exp(-a.lambda[k] * t);
        double sx, cx, sy, cy;
        sincos(kx * x, &sx, &cx);
        sincos(ky * y, &sy, &cy);
        const double gx = 1.0 - cx, gy = 1.0 - cy;
        u += e * gx * gy;
        ut -= a.lambda[k] * e * gx * gy;
        ux += e * kx * sx * gy;
        uy += e * gx * ky * sy;
        uxx += e * kx * kx * cx * gy;
        uyy += e * gx * ky * ky * cy;
    }
    const double lap = uxx + uyy;
    const double u2 = u * u;
    const double N = a.c_chi * a.T_amb + a.c_rad * (a.T_amb4 - u2 * u2) +
                     a.C_nld * (u2 * u * lap + 3.0 * u2 * (ux * ux + uy * uy));
    return ut - a.C_d * lap + a.c_W * (a.wind_x * ux + a.wind_y * uy) + a.c_chi * u - N;
}

// one thread per DOF (i, j): sum over the (p+1)^2 elements of its support and their q^2 points
template <typename P>
__global__ void k_forcing(MmsArgs a, P* out1, P s1, P* out2, P s2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= a.Nx || j >= a.Ny) return;
    const int p = a.p, q = a.q, NB = p + 1;
    const double t = *a.t;
    double acc = 0.0;
    for (int ey = j - p; ey <= j; ++ey) {
        if (ey < 0 || ey >= a.ny) continue;
        const int l = j - ey;
        for (int ex = i - p; ex <= i; ++ex) {
            if (ex < 0 || ex >= a.nx) continue;
            const int k = i - ex;
            for (int b = 0; b < q; ++b) {
                const double y = (ey + a.xi[b]) * a.hy;
                const double wy = a.w[b] * a.hy * a.By[((size_t)ey * q + b) * NB + l];
                for (int c = 0; c < q; ++c) {
                    const double x = (ex + a.xi[c]) * a.hx;
                    const double wx = a.w[c] * a.hx * a.Bx[((size_t)ex * q + c) * NB + k];
                    acc += wy * wx * mms_forcing(a, x, y, t);
                }
            }
        }
    }
    const size_t g = (size_t)j * a.pitch + i;
    out1[g] += s1 * (P)acc;
    if (out2) out2[g] += s2 * (P)acc;
}

__global__ void k_advance_time(double* t, double dt) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *t += dt;
}

}  // namespace

cudaError_t launch_forcing(int prec, const MmsArgs& a, void* out1, double s1, void* out2, double s2,
                           cudaStream_t s) {
    dim3 block(32, 4), grid((a.Nx + 31) / 32, (a.Ny + 3) / 4);
    if (prec == 0)
        k_forcing<float><<<grid, block, 0, s>>>(a, (float*)out1, (float)s1, (float*)out2, (float)s2);
    else
        k_forcing<double><<<grid, block, 0, s>>>(a, (double*)out1, s1, (double*)out2, s2);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_advance_time(double* t, double dt, cudaStream_t s) {
    k_advance_time<<<1, 32, 0, s>>>(t, dt);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace wf
