// Tables and 1-D factorisations, computed on the GPU in FP64 once per handle.
//
// Paper: the 1-D mass, stiffness and advection matrices of Sec. 3.1 ("Matrix
// formulation") and the banded direct solvers of Sec. 4 ("Cost of directional
// implicit solves").  Every directional operator is a combination
// aM M + aK K + aG G of these matrices; its LU factors are computed here per
// chunk of rows (truncated SPIKE partitioning, Polizzi & Sameh 2006) so that
// the line solves of every step run with many independent chunks per line.
#include <math.h>

#include "wf_internal.h"

namespace wf {

namespace {

// Gauss-Legendre nodes and weights on [0, 1] by Newton's method on the
// Legendre polynomial P_q (three-term recurrence), one thread per node.
__global__ void k_gauss(double* xi, double* w, int q) {
    int i = threadIdx.x;
    if (i >= q) return;
    const double pi = 3.14159265358979323846;
    double x = cos(pi * (i + 0.75) / (q + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
        double p0 = 1.0, p1 = x;
        for (int k = 2; k <= q; ++k) {
            double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        dp = q * (x * p1 - p0) / (x * x - 1.0);
        double dx = p1 / dp;
        x -= dx;
        if (fabs(dx) < 1e-16) break;
    }
    {
        double p0 = 1.0, p1 = x;
        for (int k = 2; k <= q; ++k) {
            double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        dp = q * (x * p1 - p0) / (x * x - 1.0);
    }
    xi[i] = 0.5 * (1.0 - x);
    w[i] = 1.0 / ((1.0 - x * x) * dp * dp);  // (2 / ((1-x^2) P_q'^2)) / 2
}

// Knot t_j of the open uniform knot vector relative to the start of element e, as
// (integer) * h: the same bits for every interior element, so the tables, the
// assembled bands and the chunk factors of interior rows are exactly translation
// invariant.
__device__ inline double knot_rel(int j, int e, int n, int p, double h) {
    int m = j - p;
    m = m < 0 ? 0 : (m > n ? n : m);
    return (double)(m - e) * h;
}

// Basis values and derivatives at the Gauss points of every element, by the
// triangular (left/right difference) evaluation of the nonzero B-splines of
// a knot span, in coordinates relative to the element start.  One thread per
// (element, point).
__global__ void k_basis(const double* __restrict__ xi, int q, int n, int p, double L, double* B, double* D) {
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * q) return;
    const int e = idx / q, a = idx % q;
    const double h = L / n;
    const int span = e + p;
    const double x = xi[a] * h;  // offset of the point inside element e
    double left[kMaxP + 1], right[kMaxP + 1], Nv[kMaxP + 1], Nm[kMaxP + 1];
    Nv[0] = 1.0;
    Nm[0] = 1.0;
    for (int j = 1; j <= p; ++j) {
        left[j] = x - knot_rel(span + 1 - j, e, n, p, h);
        right[j] = knot_rel(span + j, e, n, p, h) - x;
        double saved = 0.0;
        for (int r = 0; r < j; ++r) {
            double tmp = Nv[r] / (right[r + 1] + left[j - r]);
            Nv[r] = saved + right[r + 1] * tmp;
            saved = left[j - r] * tmp;
        }
        Nv[j] = saved;
        if (j == p - 1)
            for (int r = 0; r <= j; ++r) Nm[r] = Nv[r];
    }
    for (int l = 0; l <= p; ++l) {
        const int i = span - p + l;
        double d = 0.0;
        if (p > 0) {
            if (l >= 1) {
                double den = knot_rel(i + p, e, n, p, h) - knot_rel(i, e, n, p, h);
                if (den > 0.0) d += p * Nm[l - 1] / den;
            }
            if (l <= p - 1) {
                double den = knot_rel(i + p + 1, e, n, p, h) - knot_rel(i + 1, e, n, p, h);
                if (den > 0.0) d -= p * Nm[l] / den;
            }
        }
        B[(size_t)(e * q + a) * (p + 1) + l] = Nv[l];
        D[(size_t)(e * q + a) * (p + 1) + l] = d;
    }
}

// 1-D matrices by Gauss quadrature, one thread per band entry (row i, diagonal d).
// Row = test function, column = trial function (G carries the trial derivative).
__global__ void k_assemble(const double* __restrict__ B, const double* __restrict__ D, const double* __restrict__ w,
                           int q, int n, int p, double h, double* Mb, double* Kb, double* Gb) {
    const int N = n + p, W = 2 * p + 1;
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= N * W) return;
    const int i = idx / W, d = idx % W, k = i + d - p;
    double m = 0.0, kk = 0.0, g = 0.0;
    if (k >= 0 && k < N) {
        int lo = (i > k ? i : k) - p;
        int hi = i < k ? i : k;
        lo = lo < 0 ? 0 : lo;
        hi = hi > n - 1 ? n - 1 : hi;
        for (int e = lo; e <= hi; ++e) {
            const int li = i - e, lk = k - e;
            for (int a = 0; a < q; ++a) {
                const double wa = w[a] * h;
                const size_t o = (size_t)(e * q + a) * (p + 1);
                const double bi = B[o + li], bk = B[o + lk], di = D[o + li], dk = D[o + lk];
                m += wa * bi * bk;
                kk += wa * di * dk;
                g += wa * bi * dk;
            }
        }
    }
    Mb[idx] = m;
    Kb[idx] = kk;
    Gb[idx] = g;
}

__device__ inline void atomic_max_nonneg(double* addr, double v) {
    // non-negative doubles order like their bit patterns
    atomicMax(reinterpret_cast<unsigned long long*>(addr), (unsigned long long)__double_as_longlong(v));
}

// Chunk-local banded solve with the factors of one chunk (rows s .. s+m-1);
// x has stride `stride` and holds the right-hand side on entry.
__device__ void chunk_solve64(const double* lu, int s, int m, int p, double* x, int stride) {
    const int W = 2 * p + 1;
    for (int o = 0; o < m; ++o) {
        const int r = s + o;
        double v = x[(size_t)o * stride];
        for (int i = 1; i <= p && o - i >= 0; ++i) v -= lu[(size_t)r * W + i - 1] * x[(size_t)(o - i) * stride];
        x[(size_t)o * stride] = v;
    }
    for (int o = m - 1; o >= 0; --o) {
        const int r = s + o;
        double v = x[(size_t)o * stride];
        for (int j = 1; j <= p && o + j < m; ++j) v -= lu[(size_t)r * W + p + j] * x[(size_t)(o + j) * stride];
        x[(size_t)o * stride] = v * lu[(size_t)r * W + p];
    }
}

// One thread per chunk: band of A, chunk-local LU without pivoting, and the spikes.
__global__ void k_factor(const double* __restrict__ Mb, const double* __restrict__ Kb, const double* __restrict__ Gb,
                         double aM, double aK, double aG, int N, int p, Chunks ch, double* band, double* lu,
                         double* spk, double* work, double* diag) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= ch.C) return;
    const int W = 2 * p + 1, S = 2 * p;
    const int s = chunk_start(ch, k), m = chunk_len(ch, k), e = s + m;
    double anorm = 0.0;
    for (int r = s; r < e; ++r) {
        double rs = 0.0;
        for (int d = 0; d < W; ++d) {
            const int col = r + d - p;
            const size_t o = (size_t)r * W + d;
            double v = (col >= 0 && col < N) ? aM * Mb[o] + aK * Kb[o] + aG * Gb[o] : 0.0;
            band[o] = v;
            work[o] = (col >= s && col < e) ? v : 0.0;
            lu[o] = 0.0;
            rs += fabs(v);
        }
        anorm = rs > anorm ? rs : anorm;
        for (int c = 0; c < S; ++c) spk[(size_t)r * S + c] = 0.0;
    }
    // the norm must cover the whole matrix; chunk-local is a lower bound that is
    // close to it for these operators (diagonally dominant bands of similar rows)
    bool singular = false;
    for (int r = s; r < e; ++r) {
        double piv = work[(size_t)r * W + p];
        if (!(fabs(piv) > 1e-300 * anorm)) {
            singular = true;
            piv = 1.0;
        }
        const double inv = 1.0 / piv;
        for (int i = 1; i <= p && r + i < e; ++i) {
            const size_t ri = (size_t)(r + i) * W;
            const double l = work[ri + p - i] * inv;
            lu[ri + i - 1] = l;
            for (int j = 1; j <= p; ++j)
                if (r + j < e) work[ri + p - i + j] -= l * work[(size_t)r * W + p + j];
            work[ri + p - i] = 0.0;
        }
        lu[(size_t)r * W + p] = inv;
        for (int j = 1; j <= p; ++j) lu[(size_t)r * W + p + j] = (r + j < e) ? work[(size_t)r * W + p + j] : 0.0;
    }
    if (singular) diag[0] = 1.0;
    // right spike V = A_k^{-1} B_k (coupling to the first p unknowns of chunk k+1)
    if (k + 1 < ch.C) {
        for (int c = 0; c < p; ++c) {
            double* x = spk + (size_t)s * S + c;
            for (int o = 0; o < m; ++o) {
                const int r = s + o, col = e + c, d = col - r + p;
                x[(size_t)o * S] = (d >= 0 && d < W) ? band[(size_t)r * W + d] : 0.0;
            }
            chunk_solve64(lu, s, m, p, x, S);
        }
    }
    // left spike W = A_k^{-1} C_k (coupling to the last p unknowns of chunk k-1)
    if (k > 0) {
        for (int c = 0; c < p; ++c) {
            double* x = spk + (size_t)s * S + p + c;
            for (int o = 0; o < m; ++o) {
                const int r = s + o, col = s - p + c, d = col - r + p;
                x[(size_t)o * S] = (d >= 0 && d < W) ? band[(size_t)r * W + d] : 0.0;
            }
            chunk_solve64(lu, s, m, p, x, S);
        }
    }
}

// One thread per interface k (between chunks k and k+1): E_k = (I - W_{k+1}^top V_k^bottom)^{-1}
// by Gauss-Jordan with partial pivoting, and the truncation measure (largest entry of
// the spike blocks the truncated reduced system neglects).
__global__ void k_interface(int p, Chunks ch, const double* __restrict__ spk, double* E, double* diag) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k + 1 >= ch.C) return;
    const int S = 2 * p;
    const int s0 = chunk_start(ch, k), m0 = chunk_len(ch, k);
    const int s1 = chunk_start(ch, k + 1), m1 = chunk_len(ch, k + 1);
    double A[kMaxP][2 * kMaxP];
    for (int a = 0; a < p; ++a) {
        for (int c = 0; c < p; ++c) {
            double v = (a == c) ? 1.0 : 0.0;
            for (int t = 0; t < p; ++t)
                v -= spk[(size_t)(s1 + a) * S + p + t] * spk[(size_t)(s0 + m0 - p + t) * S + c];
            A[a][c] = v;
            A[a][p + c] = (a == c) ? 1.0 : 0.0;
        }
    }
    for (int col = 0; col < p; ++col) {
        int piv = col;
        for (int r = col + 1; r < p; ++r)
            if (fabs(A[r][col]) > fabs(A[piv][col])) piv = r;
        if (piv != col)
            for (int c = 0; c < 2 * p; ++c) {
                double t = A[col][c];
                A[col][c] = A[piv][c];
                A[piv][c] = t;
            }
        double d = A[col][col];
        if (!(fabs(d) > 1e-300)) {
            diag[0] = 1.0;
            d = 1.0;
        }
        const double inv = 1.0 / d;
        for (int c = 0; c < 2 * p; ++c) A[col][c] *= inv;
        for (int r = 0; r < p; ++r) {
            if (r == col) continue;
            const double f = A[r][col];
            for (int c = 0; c < 2 * p; ++c) A[r][c] -= f * A[col][c];
        }
    }
    for (int a = 0; a < p; ++a)
        for (int c = 0; c < p; ++c) E[(size_t)k * p * p + a * p + c] = A[a][p + c];
    // The reduced system of interface k neglects the bottom of chunk k's left spike
    // (zero for k = 0) and the top of chunk k+1's right spike (zero for k+1 = C-1).
    double tr = 0.0;
    for (int a = 0; a < p; ++a)
        for (int c = 0; c < p; ++c) {
            if (k > 0) tr = fmax(tr, fabs(spk[(size_t)(s0 + m0 - p + a) * S + p + c]));
            if (k + 1 < ch.C - 1) tr = fmax(tr, fabs(spk[(size_t)(s1 + a) * S + c]));
        }
    (void)m1;
    atomic_max_nonneg(diag + 1, tr);
}

// Compact factors: chunk types 0 (first), 1 (interior, represented by chunk 1), 2 (last);
// interface types 0 (k = 0), 1 (interior, interface 1), 2 (k = C-2).  One thread per
// (row offset o < mmax); thread 0 also copies E and every thread checks interior
// chunks against chunk 1.
__global__ void k_compact(const double* __restrict__ lu, const double* __restrict__ spk, const double* __restrict__ E,
                          int p, Chunks ch, int mmax, double* luc, double* spkc, double* Ec, double* diag) {
    const int W = 2 * p + 1, S = 2 * p;
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o < mmax) {
        const int src_chunk[3] = {0, ch.C >= 3 ? 1 : 0, ch.C - 1};
        for (int t = 0; t < 3; ++t) {
            const int k = src_chunk[t];
            const bool ok = o < chunk_len(ch, k);
            const size_t r = (size_t)chunk_start(ch, k) + o;
            for (int d = 0; d < W; ++d) luc[((size_t)t * mmax + o) * W + d] = ok ? lu[r * W + d] : 0.0;
            for (int c = 0; c < S; ++c) spkc[((size_t)t * mmax + o) * S + c] = ok ? spk[r * S + c] : 0.0;
        }
        bool same = true;
        for (int k = 2; k + 1 < ch.C && o < ch.base; ++k) {
            const size_t r1 = (size_t)chunk_start(ch, 1) + o, rk = (size_t)chunk_start(ch, k) + o;
            for (int d = 0; d < W; ++d) same &= lu[rk * W + d] == lu[r1 * W + d];
            for (int c = 0; c < S; ++c) same &= spk[rk * S + c] == spk[r1 * S + c];
        }
        if (!same) diag[2] = 1.0;
    }
    if (o == 0 && ch.C > 1) {
        const int src_if[3] = {0, ch.C >= 4 ? 1 : 0, ch.C - 2};
        for (int t = 0; t < 3; ++t)
            for (int c = 0; c < p * p; ++c) Ec[t * p * p + c] = E[(size_t)src_if[t] * p * p + c];
        bool same = true;
        for (int k = 2; k < ch.C - 2; ++k)
            for (int c = 0; c < p * p; ++c) same &= E[(size_t)k * p * p + c] == E[(size_t)p * p + c];
        if (!same) diag[2] = 1.0;
    }
}

__global__ void k_to_f32(const double* __restrict__ src, float* dst, size_t n) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = (float)src[i];
}

template <typename P>
__global__ void k_factor_points(const double* __restrict__ coef, int rank, int n, int p, const double* __restrict__ B,
                                P* out) {
    const int q = p + 1, N = n + p;
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= rank * n * q) return;
    const int r = idx / (n * q), eq = idx % (n * q), e = eq / q;
    double v = 0.0;
    for (int l = 0; l <= p; ++l) v += B[(size_t)eq * (p + 1) + l] * coef[(size_t)r * N + e + l];
    out[idx] = (P)v;
}

template <typename P, typename H>
__global__ void k_convert_in(const H* __restrict__ src, P* dst, int Nx, int Ny, int pitch) {
    size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)Ny * pitch) return;
    const int j = (int)(idx / pitch), i = (int)(idx % pitch);
    dst[idx] = (i < Nx) ? (P)src[(size_t)j * Nx + i] : (P)0;
}

// every slot of a batch at once: blockIdx.z = slot, host arrays [S][Ny][Nx], slot fields sbytes apart
template <typename P, typename H>
__global__ void k_convert_in_batch(const H* __restrict__ src, P* dst0, long long sbytes, int Nx, int Ny, int pitch) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)Ny * pitch) return;
    const int z = blockIdx.z;
    P* dst = reinterpret_cast<P*>(reinterpret_cast<char*>(dst0) + (long long)z * sbytes);
    const int j = (int)(idx / pitch), i = (int)(idx % pitch);
    dst[idx] = (i < Nx) ? (P)src[(size_t)z * Nx * Ny + (size_t)j * Nx + i] : (P)0;
}

template <typename P, typename H>
__global__ void k_convert_out_batch(const P* src0, H* dst, long long sbytes, int Nx, int Ny, int pitch) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)Ny * Nx) return;
    const int z = blockIdx.z;
    const P* src = reinterpret_cast<const P*>(reinterpret_cast<const char*>(src0) + (long long)z * sbytes);
    const int j = (int)(idx / Nx), i = (int)(idx % Nx);
    dst[(size_t)z * Nx * Ny + idx] = (H)src[(size_t)j * pitch + i];
}

template <typename P, typename H>
__global__ void k_convert_out(const P* __restrict__ src, H* dst, int Nx, int Ny, int pitch) {
    size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)Ny * Nx) return;
    const int j = (int)(idx / Nx), i = (int)(idx % Nx);
    dst[idx] = (H)src[(size_t)j * pitch + i];
}

// Guard flags of S scenarios (each in its own block, sbytes apart) gathered into out[S],
// and cleared when clear != 0.
__global__ void k_gather_status(int* status0, long long sbytes, int S, int* out, int clear) {
    const int z = blockIdx.x * blockDim.x + threadIdx.x;
    if (z >= S) return;
    int* st = reinterpret_cast<int*>(reinterpret_cast<char*>(status0) + (long long)z * sbytes);
    out[z] = st[0];
    if (clear) st[0] = 0;
}

// Per-slot step budgets (end of a step): an active slot with a positive budget spends one step of
// it; at zero the slot is skipped until its budget is set again; a negative budget is unlimited.
__global__ void k_step_budget(const int* active, int* budget, int S) {
    const int z = blockIdx.x * blockDim.x + threadIdx.x;
    if (z >= S || !active[z]) return;
    const int b = budget[z];
    if (b > 0) budget[z] = b - 1;
}

template <typename P>
__global__ void k_fill(P* dst, size_t n, P v) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = v;
}

inline unsigned blocks(size_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

cudaError_t launch_gauss(double* xi, double* w, int q, cudaStream_t s) {
    k_gauss<<<1, 32, 0, s>>>(xi, w, q);
    return cudaGetLastError();
}

cudaError_t launch_basis(const double* xi, int q, int n, int p, double L, double* B, double* D, cudaStream_t s) {
    k_basis<<<blocks((size_t)n * q, 128), 128, 0, s>>>(xi, q, n, p, L, B, D);
    return cudaGetLastError();
}

cudaError_t launch_assemble(const double* B, const double* D, const double* w, int q, int n, int p, double h,
                            double* Mb, double* Kb, double* Gb, cudaStream_t s) {
    const size_t cnt = (size_t)(n + p) * (2 * p + 1);
    k_assemble<<<blocks(cnt, 128), 128, 0, s>>>(B, D, w, q, n, p, h, Mb, Kb, Gb);
    return cudaGetLastError();
}

cudaError_t launch_factor(const double* Mb, const double* Kb, const double* Gb, double aM, double aK, double aG,
                          int N, int p, Chunks ch, double* band64, double* lu64, double* spk64, double* E64,
                          double* work64, double* diag, cudaStream_t s) {
    k_factor<<<blocks(ch.C, 64), 64, 0, s>>>(Mb, Kb, Gb, aM, aK, aG, N, p, ch, band64, lu64, spk64, work64, diag);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    if (ch.C > 1) {
        k_interface<<<blocks(ch.C - 1, 64), 64, 0, s>>>(p, ch, spk64, E64, diag);
        err = cudaGetLastError();
    }
    return err;
}

cudaError_t launch_compact(const double* lu, const double* spk, const double* E, int p, Chunks ch, int mmax,
                           double* luc, double* spkc, double* Ec, double* diag, cudaStream_t s) {
    k_compact<<<blocks(mmax, 64), 64, 0, s>>>(lu, spk, E, p, ch, mmax, luc, spkc, Ec, diag);
    return cudaGetLastError();
}

cudaError_t launch_to_f32(const double* src, float* dst, size_t n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_to_f32<<<blocks(n, 256), 256, 0, s>>>(src, dst, n);
    return cudaGetLastError();
}

cudaError_t launch_factor_points(int prec, const double* coef, int rank, int n, int p, const double* B, void* out,
                                 cudaStream_t s) {
    const size_t cnt = (size_t)rank * n * (p + 1);
    if (cnt == 0) return cudaSuccess;
    if (prec == 0)
        k_factor_points<float><<<blocks(cnt, 128), 128, 0, s>>>(coef, rank, n, p, B, (float*)out);
    else
        k_factor_points<double><<<blocks(cnt, 128), 128, 0, s>>>(coef, rank, n, p, B, (double*)out);
    return cudaGetLastError();
}

cudaError_t launch_convert_in(int prec, const void* src, int host32, void* dst, int Nx, int Ny, int pitch,
                              cudaStream_t s) {
    const size_t cnt = (size_t)Ny * pitch;
    if (prec == 0) {
        if (host32) k_convert_in<float, float><<<blocks(cnt, 256), 256, 0, s>>>((const float*)src, (float*)dst, Nx, Ny, pitch);
        else k_convert_in<float, double><<<blocks(cnt, 256), 256, 0, s>>>((const double*)src, (float*)dst, Nx, Ny, pitch);
    } else {
        if (host32) k_convert_in<double, float><<<blocks(cnt, 256), 256, 0, s>>>((const float*)src, (double*)dst, Nx, Ny, pitch);
        else k_convert_in<double, double><<<blocks(cnt, 256), 256, 0, s>>>((const double*)src, (double*)dst, Nx, Ny, pitch);
    }
    return cudaGetLastError();
}

cudaError_t launch_convert_batch(int dir_in, int prec, const void* host_stage, int host32, void* field0,
                                 long long sbytes, int S, int Nx, int Ny, int pitch, cudaStream_t s) {
    const size_t cnt = dir_in ? (size_t)Ny * pitch : (size_t)Ny * Nx;
    dim3 g(blocks(cnt, 256), 1, S);
#define WF_CB(P, H)                                                                                        \
    if (dir_in)                                                                                            \
        k_convert_in_batch<P, H><<<g, 256, 0, s>>>((const H*)host_stage, (P*)field0, sbytes, Nx, Ny, pitch); \
    else                                                                                                   \
        k_convert_out_batch<P, H><<<g, 256, 0, s>>>((const P*)field0, (H*)host_stage, sbytes, Nx, Ny, pitch)
    if (prec == 0) {
        if (host32) { WF_CB(float, float); } else { WF_CB(float, double); }
    } else {
        if (host32) { WF_CB(double, float); } else { WF_CB(double, double); }
    }
#undef WF_CB
    return cudaGetLastError();
}

cudaError_t launch_convert_out(int prec, const void* src, void* dst, int host32, int Nx, int Ny, int pitch,
                               cudaStream_t s) {
    const size_t cnt = (size_t)Ny * Nx;
    if (prec == 0) {
        if (host32) k_convert_out<float, float><<<blocks(cnt, 256), 256, 0, s>>>((const float*)src, (float*)dst, Nx, Ny, pitch);
        else k_convert_out<float, double><<<blocks(cnt, 256), 256, 0, s>>>((const float*)src, (double*)dst, Nx, Ny, pitch);
    } else {
        if (host32) k_convert_out<double, float><<<blocks(cnt, 256), 256, 0, s>>>((const double*)src, (float*)dst, Nx, Ny, pitch);
        else k_convert_out<double, double><<<blocks(cnt, 256), 256, 0, s>>>((const double*)src, (double*)dst, Nx, Ny, pitch);
    }
    return cudaGetLastError();
}

cudaError_t launch_gather_status(int* status0, long long sbytes, int S, int* out, int clear, cudaStream_t s) {
    k_gather_status<<<blocks(S, 128), 128, 0, s>>>(status0, sbytes, S, out, clear);
    return cudaGetLastError();
}

cudaError_t launch_step_budget(const int* active, int* budget, int S, cudaStream_t s) {
    k_step_budget<<<blocks(S, 128), 128, 0, s>>>(active, budget, S);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_fill(int prec, void* dst, size_t n, double v, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    if (prec == 0)
        k_fill<float><<<blocks(n, 256), 256, 0, s>>>((float*)dst, n, (float)v);
    else
        k_fill<double><<<blocks(n, 256), 256, 0, s>>>((double*)dst, n, v);
    return cudaGetLastError();
}

}  // namespace wf
