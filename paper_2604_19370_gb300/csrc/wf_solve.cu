// Independent 1-D banded solves along x and along y (shared-memory form).
//
// Paper: Sec. 4 ("Cost of directional implicit solves"): a system
// (A^x (x) B^y) X = R is solved as N_y independent solves of size N_x with
// A^x and N_x independent solves of size N_y with B^y, each banded with
// half-bandwidth p (O(p^2 N) in total).
//
// GPU form: every line is cut into C chunks (truncated SPIKE, Polizzi & Sameh
// 2006).  One thread owns one chunk of one line: it runs the chunk-local LU
// forward/backward substitution, the threads of neighbouring chunks exchange
// their p boundary values through shared memory to solve the p x p interface
// systems, and each thread subtracts the spike corrections.  The neglected
// coupling decays geometrically with the chunk length and is checked against
// a tolerance when the factors are built.
//
// x pass: a CTA owns ROWS consecutive rows; their full length is staged in
// shared memory with coalesced row loads and stores (rows are contiguous).
// y pass: a CTA owns COLS consecutive columns; neighbouring lanes hold
// neighbouring columns, so every global load and store is a contiguous run
// of COLS elements (one 32-byte sector) per chunk.
#include "wf_internal.h"

namespace wf {

namespace {

template <typename P>
struct FactorT {
    Chunks ch;
    const P* __restrict__ lu;
    const P* __restrict__ spk;
    const P* __restrict__ E;
};

template <typename P>
FactorT<P> typed(const FactorV& f) {
    FactorT<P> t;
    t.ch = f.ch;
    t.lu = (const P*)f.lu;
    t.spk = (const P*)f.spk;
    t.E = (const P*)f.E;
    return t;
}

template <typename P>
struct LineArgsT {
    int nlines, pitch, mpad;
    const P* in[2];
    P* out[2];
    FactorT<P> f[2];
    const P* premul[2];
    P prescale[2];
    const P* base[2];
    int* status;
    P tmax;
    Batch b;
};

template <typename P>
__device__ __forceinline__ LineArgsT<P> scene_line_args(const LineArgsT<P>& a_in) {
    LineArgsT<P> a = a_in;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        a.in[q] = scene_ptr(a.in[q], a.b);
        a.out[q] = scene_ptr(a.out[q], a.b);
        a.f[q].lu = scene_ptr(a.f[q].lu, a.b);
        a.f[q].spk = scene_ptr(a.f[q].spk, a.b);
        a.f[q].E = scene_ptr(a.f[q].E, a.b);
        a.premul[q] = scene_ptr(a.premul[q], a.b);
        a.base[q] = scene_ptr(a.base[q], a.b);
    }
    a.status = scene_ptr(a.status, a.b);
    return a;
}

// Forward and backward substitution of one chunk, in place on g (stride 1).
template <typename P, int PD>
__device__ __forceinline__ void chunk_lu_solve(P* g, int m, const P* __restrict__ lu) {
    constexpr int W = 2 * PD + 1;
    P prev[PD];
#pragma unroll
    for (int i = 0; i < PD; ++i) prev[i] = P(0);
    for (int o = 0; o < m; ++o) {
        P v = g[o];
#pragma unroll
        for (int i = 0; i < PD; ++i) v -= lu[(size_t)o * W + i] * prev[i];
#pragma unroll
        for (int i = PD - 1; i > 0; --i) prev[i] = prev[i - 1];
        prev[0] = v;
        g[o] = v;
    }
#pragma unroll
    for (int i = 0; i < PD; ++i) prev[i] = P(0);
    for (int o = m - 1; o >= 0; --o) {
        P v = g[o];
#pragma unroll
        for (int j = 0; j < PD; ++j) v -= lu[(size_t)o * W + PD + 1 + j] * prev[j];
        v *= lu[(size_t)o * W + PD];
#pragma unroll
        for (int j = PD - 1; j > 0; --j) prev[j] = prev[j - 1];
        prev[0] = v;
        g[o] = v;
    }
}

// Interface unknowns of chunk k: tn = first PD values of chunk k+1, bp = last PD values of chunk k-1.
// g, gn, gp: local solutions of chunks k, k+1, k-1 (stride 1).
template <typename P, int PD>
__device__ __forceinline__ void interface_values(const FactorT<P>& f, int k, const P* g, int m, const P* gn,
                                                 const P* gp, P* tn, P* bp) {
    constexpr int S = 2 * PD;
    const Chunks& ch = f.ch;
#pragma unroll
    for (int a = 0; a < PD; ++a) tn[a] = bp[a] = P(0);
    if (k + 1 < ch.C) {
        const int s1 = chunk_start(ch, k + 1);
        const P* E = f.E + (size_t)k * PD * PD;
        P rhs[PD];
#pragma unroll
        for (int a = 0; a < PD; ++a) {
            P v = gn[a];
#pragma unroll
            for (int c = 0; c < PD; ++c) v -= f.spk[(size_t)(s1 + a) * S + PD + c] * g[m - PD + c];
            rhs[a] = v;
        }
#pragma unroll
        for (int a = 0; a < PD; ++a) {
            P v = 0;
#pragma unroll
            for (int c = 0; c < PD; ++c) v += E[a * PD + c] * rhs[c];
            tn[a] = v;
        }
    }
    if (k > 0) {
        const int s = chunk_start(ch, k);
        const int sp = chunk_start(ch, k - 1), mp = chunk_len(ch, k - 1);
        const P* E = f.E + (size_t)(k - 1) * PD * PD;
        P rhs[PD], tk[PD];
#pragma unroll
        for (int a = 0; a < PD; ++a) {
            P v = g[a];
#pragma unroll
            for (int c = 0; c < PD; ++c) v -= f.spk[(size_t)(s + a) * S + PD + c] * gp[mp - PD + c];
            rhs[a] = v;
        }
#pragma unroll
        for (int a = 0; a < PD; ++a) {
            P v = 0;
#pragma unroll
            for (int c = 0; c < PD; ++c) v += E[a * PD + c] * rhs[c];
            tk[a] = v;
        }
#pragma unroll
        for (int a = 0; a < PD; ++a) {
            P v = gp[mp - PD + a];
#pragma unroll
            for (int c = 0; c < PD; ++c) v -= f.spk[(size_t)(sp + mp - PD + a) * S + c] * tk[c];
            bp[a] = v;
        }
    }
}

template <typename P, int PD>
__device__ __forceinline__ P spike_correct(const P* __restrict__ sk, P g, const P* tn, const P* bp) {
    constexpr int S = 2 * PD;
#pragma unroll
    for (int c = 0; c < PD; ++c) g -= sk[c] * tn[c] + sk[PD + c] * bp[c];
    (void)S;
    return g;
}

// x pass.  blockIdx.x: group of ROWS rows; blockIdx.y: array.  blockDim.x = ROWS * C.
template <typename P, int PD, int ROWS>
__global__ void k_xsolve(const LineArgsT<P> a_in) {
    if (!scene_active(a_in.b)) return;
    const LineArgsT<P> a = scene_line_args(a_in);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    P* buf = reinterpret_cast<P*>(smem_raw);
    const int arr = blockIdx.y;
    const P* __restrict__ in = a.in[arr];
    P* out = a.out[arr];
    const FactorT<P> f = a.f[arr];
    const Chunks ch = f.ch;
    const int N = ch.N, mpad = a.mpad;
    const int j0 = blockIdx.x * ROWS;
    const int tid = threadIdx.x, nt = blockDim.x;

    for (int idx = tid; idx < ROWS * N; idx += nt) {
        const int r = idx / N, x = idx - r * N;
        const int k = chunk_of(ch, x);
        const int j = j0 + r;
        buf[(k * ROWS + r) * mpad + (x - chunk_start(ch, k))] = (j < a.nlines) ? in[(size_t)j * a.pitch + x] : P(0);
    }
    __syncthreads();

    const int k = tid / ROWS, r = tid - k * ROWS;
    const int s = chunk_start(ch, k), m = chunk_len(ch, k);
    P* g = buf + (size_t)tid * mpad;
    chunk_lu_solve<P, PD>(g, m, f.lu + (size_t)s * (2 * PD + 1));
    __syncthreads();

    P tn[PD], bp[PD];
    const P* gn = (k + 1 < ch.C) ? buf + (size_t)((k + 1) * ROWS + r) * mpad : g;
    const P* gp = (k > 0) ? buf + (size_t)((k - 1) * ROWS + r) * mpad : g;
    interface_values<P, PD>(f, k, g, m, gn, gp, tn, bp);
    __syncthreads();

    const P* sk = f.spk + (size_t)s * 2 * PD;
    for (int o = 0; o < m; ++o) g[o] = spike_correct<P, PD>(sk + (size_t)o * 2 * PD, g[o], tn, bp);
    __syncthreads();

    for (int idx = tid; idx < ROWS * N; idx += nt) {
        const int rr = idx / N, x = idx - rr * N;
        const int kk = chunk_of(ch, x);
        const int j = j0 + rr;
        if (j < a.nlines) out[(size_t)j * a.pitch + x] = buf[(kk * ROWS + rr) * mpad + (x - chunk_start(ch, kk))];
    }
}

// y pass.  blockIdx.x: group of COLS columns; blockIdx.y: array.  blockDim.x = COLS * C.
template <typename P, int PD, int COLS>
__global__ void k_ysolve(const LineArgsT<P> a_in) {
    if (!scene_active(a_in.b)) return;
    const LineArgsT<P> a = scene_line_args(a_in);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    P* buf = reinterpret_cast<P*>(smem_raw);
    constexpr int W = 2 * PD + 1;
    const int arr = blockIdx.y;
    const P* in = a.in[arr];
    P* out = a.out[arr];
    const P* __restrict__ pre = a.premul[arr];
    const P prescale = a.prescale[arr];
    const P* base = a.base[arr];
    const FactorT<P> f = a.f[arr];
    const Chunks ch = f.ch;
    const int N = ch.N, mpad = a.mpad;
    const int tid = threadIdx.x;
    const int k = tid / COLS, c = tid - k * COLS;
    const int i = blockIdx.x * COLS + c;
    const bool valid = i < a.nlines;
    const int s = chunk_start(ch, k), m = chunk_len(ch, k);
    P* g = buf + (size_t)tid * mpad;

    if (valid) {
        if (pre) {
            for (int o = 0; o < m; ++o) {
                const int row = s + o;
                P v = 0;
#pragma unroll
                for (int d = 0; d < W; ++d) {
                    const int rr = row + d - PD;
                    if (rr >= 0 && rr < N) v += pre[(size_t)row * W + d] * in[(size_t)rr * a.pitch + i];
                }
                g[o] = prescale * v;
            }
        } else {
            for (int o = 0; o < m; ++o) g[o] = in[(size_t)(s + o) * a.pitch + i];
        }
    } else {
        for (int o = 0; o < m; ++o) g[o] = P(0);
    }
    chunk_lu_solve<P, PD>(g, m, f.lu + (size_t)s * W);
    __syncthreads();

    P tn[PD], bp[PD];
    const P* gn = (k + 1 < ch.C) ? buf + (size_t)((k + 1) * COLS + c) * mpad : g;
    const P* gp = (k > 0) ? buf + (size_t)((k - 1) * COLS + c) * mpad : g;
    interface_values<P, PD>(f, k, g, m, gn, gp, tn, bp);
    __syncthreads();

    if (!valid) return;
    const P* sk = f.spk + (size_t)s * 2 * PD;
    bool bad = false;
    const bool guard = (a.status != nullptr) && arr == 0;
    for (int o = 0; o < m; ++o) {
        const size_t gi = (size_t)(s + o) * a.pitch + i;
        P v = spike_correct<P, PD>(sk + (size_t)o * 2 * PD, g[o], tn, bp);
        if (base) v += base[gi];
        out[gi] = v;
        if (guard) bad |= !(fabs((double)v) <= (double)a.tmax);  // also catches NaN
    }
    if (guard && bad) atomicOr(a.status, 1);
}

template <typename P>
LineArgsT<P> to_typed(const LineArgs& a, int mpad) {
    LineArgsT<P> t;
    t.nlines = a.nlines;
    t.pitch = a.pitch;
    t.mpad = mpad;
    for (int q = 0; q < 2; ++q) {
        t.in[q] = (const P*)a.in[q];
        t.out[q] = (P*)a.out[q];
        t.f[q] = typed<P>(a.f[q]);
        t.premul[q] = (const P*)a.premul[q];
        t.prescale[q] = (P)a.prescale[q];
        t.base[q] = (const P*)a.base[q];
    }
    t.status = a.status;
    t.tmax = (P)a.tmax;
    t.b = a.b;
    return t;
}

inline int mpad_of(const Chunks& ch) { return (ch.base > ch.last ? ch.base : ch.last) | 1; }

template <typename P>
constexpr int lanes_per_line() { return sizeof(P) == 4 ? 8 : 4; }

template <typename P, int PD, bool X>
cudaError_t run_line(const LineArgs& a, cudaStream_t s) {
    constexpr int G = lanes_per_line<P>();
    const Chunks& ch = a.f[0].ch;
    const int mpad = mpad_of(ch);
    const int threads = G * ch.C;
    const size_t smem = (size_t)threads * mpad * sizeof(P);
    if (threads > 1024 || smem > 227 * 1024) return cudaErrorInvalidConfiguration;
    dim3 grid((a.nlines + G - 1) / G, a.narr, a.b.S);
    if (X) {
        auto kern = k_xsolve<P, PD, G>;
        cudaError_t e = allow_dynamic_smem(kern, (size_t)smem);
        if (e != cudaSuccess) return e;
        kern<<<grid, threads, smem, s>>>(to_typed<P>(a, mpad));
    } else {
        auto kern = k_ysolve<P, PD, G>;
        cudaError_t e = allow_dynamic_smem(kern, (size_t)smem);
        if (e != cudaSuccess) return e;
        kern<<<grid, threads, smem, s>>>(to_typed<P>(a, mpad));
    }
    count_launches(1);
    return cudaGetLastError();
}

template <bool X>
cudaError_t dispatch_line(int prec, int p, const LineArgs& a, cudaStream_t s) {
    if (prec == 0) {
        switch (p) {
            case 1: return run_line<float, 1, X>(a, s);
            case 2: return run_line<float, 2, X>(a, s);
            case 3: return run_line<float, 3, X>(a, s);
        }
    } else {
        switch (p) {
            case 1: return run_line<double, 1, X>(a, s);
            case 2: return run_line<double, 2, X>(a, s);
            case 3: return run_line<double, 3, X>(a, s);
        }
    }
    return cudaErrorInvalidValue;
}

}  // namespace

// The compact-factor kernels (wf_linefast.cu) take every operator whose interior chunks are
// identical and whose lines fit one CTA of 256 threads; everything else runs the kernels above.
cudaError_t launch_xsolve(int prec, int p, const LineArgs& a, cudaStream_t s) {
    cudaError_t e = launch_line_fast(prec, p, true, a, s);
    if (e != cudaErrorNotSupported) return e;
    cudaGetLastError();
    if (a.preT) return cudaErrorNotSupported;  // fused input only in the compact-factor kernel
    return dispatch_line<true>(prec, p, a, s);
}
cudaError_t launch_ysolve(int prec, int p, const LineArgs& a, cudaStream_t s) {
    cudaError_t e = launch_line_fast(prec, p, false, a, s);
    if (e != cudaErrorNotSupported) return e;
    cudaGetLastError();
    return dispatch_line<false>(prec, p, a, s);
}

int line_rows_per_cta(int prec) { return prec == 0 ? 8 : 4; }

size_t line_smem_bytes(int prec, const Chunks& ch) {
    const int G = line_rows_per_cta(prec);
    return (size_t)G * ch.C * ((ch.base > ch.last ? ch.base : ch.last) | 1) * (prec == 0 ? 4 : 8);
}

}  // namespace wf
