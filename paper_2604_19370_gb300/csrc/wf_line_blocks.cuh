// Building blocks of the chunked line solves (truncated SPIKE with compact factors in shared
// memory; Sec. 4), shared by the per-pass kernels (wf_linefast.cu) and the persistent step
// kernel (wf_persist.cu).  The scheme is described at the top of wf_linefast.cu.
#pragma once
#include "wf_internal.h"

namespace wf {

namespace {

template <typename P>
struct FastArgs {
    int nlines, pitch, mpad, G;
    int lsh;  // x pass: log2 of the lanes per line (5: one line per warp; 4: two; 3: four)
    int sp;   // x pass: row stride of the staged rows in shared memory (elements)
    int tsp;  // x pass with preT: row stride of the staged T* rows (data at column offset 4)
    Chunks ch;
    const P* in[2];
    P* out[2];
    const P* base[2];
    const P* premul[2];
    P prescale[2];
    const P* luc[2];
    const P* spkc[2];
    const P* Ec[2];
    const P* fpad[2];   // padded factor blocks (FacSmem layout), or NULL: staged element by element
    int* status;
    int* tstatus;       // x pass: bit 4 set when the staging wait gave up
    long long wait_ns;  // x pass: limit of the staging wait
    P tmax;
    int tma;  // x pass: rows staged with bulk copies (16-byte aligned rows)
    Batch b;
    const P* preT;
    const P* preF;
    P preFscale, pc1, pc2;
    const P *pA1, *pB1, *pA2, *pB2;
};

// Pointers of one array (blockIdx.y) of one scenario (blockIdx.z).  They are selected with
// conditional moves rather than by indexing the parameter arrays, which would put a copy of
// the whole argument block in local memory.
template <typename P>
struct LineView {
    const P* in;
    P* out;
    const P* base;
    const P* premul;
    P prescale;
    const P *luc, *spkc, *Ec, *fpad;
    int* status;
    int* tstatus;
    const P *preT, *preF, *pA1, *pB1, *pA2, *pB2;
};

template <typename P>
__device__ __forceinline__ LineView<P> scene_line(const FastArgs<P>& a, int arr) {
    const bool one = arr != 0;
    LineView<P> v;
    v.in = scene_ptr(one ? a.in[1] : a.in[0], a.b);
    v.out = scene_ptr(one ? a.out[1] : a.out[0], a.b);
    v.base = scene_ptr(one ? a.base[1] : a.base[0], a.b);
    v.premul = scene_ptr(one ? a.premul[1] : a.premul[0], a.b);
    v.prescale = one ? a.prescale[1] : a.prescale[0];
    v.luc = scene_ptr(one ? a.luc[1] : a.luc[0], a.b);
    v.spkc = scene_ptr(one ? a.spkc[1] : a.spkc[0], a.b);
    v.Ec = scene_ptr(one ? a.Ec[1] : a.Ec[0], a.b);
    v.fpad = scene_ptr(one ? a.fpad[1] : a.fpad[0], a.b);
    v.status = scene_ptr(a.status, a.b);
    v.tstatus = scene_ptr(a.tstatus, a.b);
    v.preT = scene_ptr(a.preT, a.b);
    v.preF = scene_ptr(a.preF, a.b);
    v.pA1 = scene_ptr(a.pA1, a.b);
    v.pB1 = scene_ptr(a.pB1, a.b);
    v.pA2 = scene_ptr(a.pA2, a.b);
    v.pB2 = scene_ptr(a.pB2, a.b);
    return v;
}

// ---- TMA bulk copies and mbarrier (PTX) ------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// global -> shared, completion signalled on the mbarrier (16-byte aligned, size multiple of 16)
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
// shared -> global, tracked by the bulk async-group of the issuing thread
__device__ __forceinline__ void bulk_store(void* dst, const void* src, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_u32(src)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit_and_wait_read() {
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Bounded mbarrier waits.  The first wait on a staging barrier gives up after the handle's wait
// limit (ns of the SM's global timer) and sets bit 4 of the slot's flag word; the kernel then
// drains the copies still in flight with a second wait of kDrainPolls polls (each try_wait may
// suspend the thread for a while), so that no copy lands in shared memory after the CTA exits.
constexpr uint32_t kDrainPolls = 1u << 20;
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// true once the barrier's phase `parity` completed; false if limit_ns passed first (limit 0: no poll)
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, long long limit_ns) {
    if (limit_ns <= 0) return false;
    const unsigned long long t0 = global_ns();
    for (uint32_t it = 0;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 15u) == 15u && (long long)(global_ns() - t0) > limit_ns) return false;
    }
}
__device__ __forceinline__ void mbar_drain(uint64_t* bar, uint32_t parity) {
    for (uint32_t it = 0; it < kDrainPolls; ++it)
        if (mbar_try_wait(bar, parity)) return;
}

// ---- factors in shared memory ---------------------------------------------------------
// Each chunk-type row of the compact factors is split into three padded vectors so that one
// row is one (or two) vector loads:
//   F[o]: L_1 .. L_p            (multipliers of rows o-1 .. o-p, forward elimination)
//   U[o]: 1/u_oo, u_o,o+1 .. u_o,o+p   (backward substitution)
//   S[o]: V_1 .. V_p, W_1 .. W_p  (spike columns)
template <int PD>
struct FacW {
    static constexpr int F = PD == 1 ? 1 : (PD == 2 ? 2 : 4);
    static constexpr int U = PD == 1 ? 2 : 4;
    static constexpr int S = PD == 1 ? 2 : (PD == 2 ? 4 : 8);
};
__host__ __device__ constexpr int round4(int n) { return (n + 3) & ~3; }
// elements of the staged factors of 3 chunk types with mmax rows (each part 16-byte aligned)
template <int PD>
__host__ __device__ constexpr int fac_elems(int mmax) {
    return round4(3 * mmax * FacW<PD>::F) + round4(3 * mmax * FacW<PD>::U) + round4(3 * mmax * FacW<PD>::S) +
           round4(3 * PD * PD);
}
template <typename P, int PD>
struct FacSmem {
    P *F, *U, *S, *E;
    __device__ __forceinline__ FacSmem(P* base, int mmax) {
        F = base;
        U = F + round4(3 * mmax * FacW<PD>::F);
        S = U + round4(3 * mmax * FacW<PD>::U);
        E = S + round4(3 * mmax * FacW<PD>::S);
    }
    __device__ __forceinline__ P* end() const { return E + round4(3 * PD * PD); }
};

// N consecutive values from a shared-memory row aligned to min(16, N * sizeof(P)) bytes
template <typename P, int N>
__device__ __forceinline__ void ldv(const P* p, P (&o)[N]) {
    if constexpr (sizeof(P) == 4 && N % 4 == 0) {
#pragma unroll
        for (int i = 0; i < N; i += 4) {
            const float4 v = *reinterpret_cast<const float4*>(p + i);
            o[i] = v.x;
            o[i + 1] = v.y;
            o[i + 2] = v.z;
            o[i + 3] = v.w;
        }
    } else if constexpr (sizeof(P) == 4 && N == 2) {
        const float2 v = *reinterpret_cast<const float2*>(p);
        o[0] = v.x;
        o[1] = v.y;
    } else if constexpr (sizeof(P) == 8 && N % 2 == 0) {
#pragma unroll
        for (int i = 0; i < N; i += 2) {
            const double2 v = *reinterpret_cast<const double2*>(p + i);
            o[i] = v.x;
            o[i + 1] = v.y;
        }
    } else {
#pragma unroll
        for (int i = 0; i < N; ++i) o[i] = p[i];
    }
}

// Forward elimination of B consecutive rows held in registers; F points at the first row's
// factors.  prev[i] holds the result i+1 rows above.
template <typename P, int PD, int B>
__device__ __forceinline__ void fwd_rows(P (&x)[B], const P* F, P (&prev)[PD]) {
    constexpr int NF = FacW<PD>::F;
    P lv[B][NF];
#pragma unroll
    for (int q = 0; q < B; ++q) ldv<P, NF>(F + q * NF, lv[q]);
#pragma unroll
    for (int q = 0; q < B; ++q) {
        P y = x[q];
#pragma unroll
        for (int i = 0; i < PD; ++i) y -= lv[q][i] * prev[i];
#pragma unroll
        for (int i = PD - 1; i > 0; --i) prev[i] = prev[i - 1];
        prev[0] = y;
        x[q] = y;
    }
}

// Backward substitution of B consecutive rows going up: x[q] is row top - q, U points at the
// factors of row top.  prev[j] holds the result j+1 rows below.
template <typename P, int PD, int B>
__device__ __forceinline__ void bwd_rows(P (&x)[B], const P* U, P (&prev)[PD]) {
    constexpr int NU = FacW<PD>::U;
    P uv[B][NU];
#pragma unroll
    for (int q = 0; q < B; ++q) ldv<P, NU>(U - q * NU, uv[q]);
#pragma unroll
    for (int q = 0; q < B; ++q) {
        P y = x[q];
#pragma unroll
        for (int j = 0; j < PD; ++j) y -= uv[q][1 + j] * prev[j];
        y *= uv[q][0];
#pragma unroll
        for (int j = PD - 1; j > 0; --j) prev[j] = prev[j - 1];
        prev[0] = y;
        x[q] = y;
    }
}

// Chunk-local forward elimination on g[0 .. m) in shared memory: batches of 8 rows whose loads
// are issued before the dependent FMA chain, then the remaining rows one by one.
template <typename P, int PD>
__device__ __forceinline__ void lu_forward(P* g, int m, const P* F) {
    constexpr int B = 8, NF = FacW<PD>::F;
    P prev[PD];
#pragma unroll
    for (int i = 0; i < PD; ++i) prev[i] = P(0);
    int o = 0;
    for (; o + B <= m; o += B) {
        P gv[B];
#pragma unroll
        for (int q = 0; q < B; ++q) gv[q] = g[o + q];
        fwd_rows<P, PD, B>(gv, F + o * NF, prev);
#pragma unroll
        for (int q = 0; q < B; ++q) g[o + q] = gv[q];
    }
    for (; o < m; ++o) {
        P gv[1] = {g[o]};
        fwd_rows<P, PD, 1>(gv, F + o * NF, prev);
        g[o] = gv[0];
    }
}

// Chunk-local backward substitution on g[0 .. m), from row m-1 up, in the same batches.
template <typename P, int PD>
__device__ __forceinline__ void lu_backward(P* g, int m, const P* U) {
    constexpr int B = 8, NU = FacW<PD>::U;
    P prev[PD];
#pragma unroll
    for (int i = 0; i < PD; ++i) prev[i] = P(0);
    int top = m - 1;
    for (; top - B + 1 >= 0; top -= B) {
        P gv[B];
#pragma unroll
        for (int q = 0; q < B; ++q) gv[q] = g[top - q];
        bwd_rows<P, PD, B>(gv, U + top * NU, prev);
#pragma unroll
        for (int q = 0; q < B; ++q) g[top - q] = gv[q];
    }
    for (; top >= 0; --top) {
        P gv[1] = {g[top]};
        bwd_rows<P, PD, 1>(gv, U + top * NU, prev);
        g[top] = gv[0];
    }
}

// Spike corrections of B consecutive rows: x[q] -= V tn + W bp with the spikes of row q at Sk.
template <typename P, int PD, int B>
__device__ __forceinline__ void spike_rows(P (&x)[B], const P* Sk, const P* tn, const P* bp) {
    constexpr int NS = FacW<PD>::S;
    P sv[B][NS];
#pragma unroll
    for (int q = 0; q < B; ++q) ldv<P, NS>(Sk + q * NS, sv[q]);
#pragma unroll
    for (int q = 0; q < B; ++q) {
#pragma unroll
        for (int r = 0; r < PD; ++r) x[q] = fma(-sv[q][r], tn[r], fma(-sv[q][PD + r], bp[r], x[q]));
    }
}

// Spike corrections on g[0 .. m) in shared memory.
template <typename P, int PD>
__device__ __forceinline__ void spike_fix(P* g, int m, const P* Sk, const P* tn, const P* bp) {
    constexpr int B = 8, NS = FacW<PD>::S;
    int o = 0;
    for (; o + B <= m; o += B) {
        P gv[B];
#pragma unroll
        for (int q = 0; q < B; ++q) gv[q] = g[o + q];
        spike_rows<P, PD, B>(gv, Sk + o * NS, tn, bp);
#pragma unroll
        for (int q = 0; q < B; ++q) g[o + q] = gv[q];
    }
    for (; o < m; ++o) {
        P gv[1] = {g[o]};
        spike_rows<P, PD, 1>(gv, Sk + o * NS, tn, bp);
        g[o] = gv[0];
    }
}

// Interface values of chunk k from its own boundary values and its neighbours':
// tn = first PD values of chunk k+1, bp = last PD values of chunk k-1 (truncated SPIKE).
template <typename P, int PD>
__device__ __forceinline__ void interface_solve(const Chunks& ch, int k, int mmax, const P* fs, const P* fe,
                                                const P* own_top, const P* own_bot, const P* nxt_top,
                                                const P* prv_bot, P* tn, P* bp) {
    constexpr int S = FacW<PD>::S;  // row stride of the staged spikes
    const int base = ch.base;
#pragma unroll
    for (int q = 0; q < PD; ++q) tn[q] = bp[q] = P(0);
    if (k + 1 < ch.C) {
        const P* Wn = fs + chunk_type(ch, k + 1) * mmax * S;
        const P* E = fe + iface_type(ch, k) * PD * PD;
        P rhs[PD];
#pragma unroll
        for (int q = 0; q < PD; ++q) {
            P x = nxt_top[q];
#pragma unroll
            for (int r = 0; r < PD; ++r) x -= Wn[q * S + PD + r] * own_bot[r];
            rhs[q] = x;
        }
#pragma unroll
        for (int q = 0; q < PD; ++q) {
            P x = 0;
#pragma unroll
            for (int r = 0; r < PD; ++r) x += E[q * PD + r] * rhs[r];
            tn[q] = x;
        }
    }
    if (k > 0) {
        const P* Wk = fs + chunk_type(ch, k) * mmax * S;
        const P* E = fe + iface_type(ch, k - 1) * PD * PD;
        const P* Vp = fs + (chunk_type(ch, k - 1) * mmax + base - PD) * S;
        P rhs[PD], tk[PD];
#pragma unroll
        for (int q = 0; q < PD; ++q) {
            P x = own_top[q];
#pragma unroll
            for (int r = 0; r < PD; ++r) x -= Wk[q * S + PD + r] * prv_bot[r];
            rhs[q] = x;
        }
#pragma unroll
        for (int q = 0; q < PD; ++q) {
            P x = 0;
#pragma unroll
            for (int r = 0; r < PD; ++r) x += E[q * PD + r] * rhs[r];
            tk[q] = x;
        }
#pragma unroll
        for (int q = 0; q < PD; ++q) {
            P x = prv_bot[q];
#pragma unroll
            for (int r = 0; r < PD; ++r) x -= Vp[q * S + r] * tk[r];
            bp[q] = x;
        }
    }
}

// Compact factors (global, [3][mmax][2p+1], [3][mmax][2p], [3][p*p]) into the padded
// shared-memory layout of FacSmem; padding entries are zero.
// (threads tid of nt stage the factors; the CTA's threads by default)
// The same layout is written once per operator into global memory (the padded factor block,
// launch_pad_factors), from where a kernel stages it with one bulk copy.
template <typename P, int PD>
__device__ __forceinline__ void fill_factors(const P* __restrict__ g1, const P* __restrict__ g2,
                                             const P* __restrict__ g3, int mmax, const FacSmem<P, PD>& fm, int tid,
                                             int nt) {
    constexpr int W = 2 * PD + 1, S2 = 2 * PD;
    constexpr int NF = FacW<PD>::F, NU = FacW<PD>::U, NS = FacW<PD>::S;
    const int rows = 3 * mmax;
    for (int i = tid; i < rows * NF; i += nt) {
        const int r = i / NF, c = i - r * NF;
        fm.F[i] = c < PD ? g1[r * W + c] : P(0);
    }
    for (int i = tid; i < rows * NU; i += nt) {
        const int r = i / NU, c = i - r * NU;
        fm.U[i] = c <= PD ? g1[r * W + PD + c] : P(0);
    }
    for (int i = tid; i < rows * NS; i += nt) {
        const int r = i / NS, c = i - r * NS;
        fm.S[i] = c < S2 ? g2[r * S2 + c] : P(0);
    }
    for (int i = tid; i < 3 * PD * PD; i += nt) fm.E[i] = g3[i];
}
template <typename P, int PD>
__device__ __forceinline__ void stage_factors(const LineView<P>& v, int mmax, const FacSmem<P, PD>& fm, int tid,
                                              int nt) {
    fill_factors<P, PD>(v.luc, v.spkc, v.Ec, mmax, fm, tid, nt);
}
template <typename P, int PD>
__device__ __forceinline__ void stage_factors(const LineView<P>& v, int mmax, const FacSmem<P, PD>& fm) {
    stage_factors<P, PD>(v, mmax, fm, threadIdx.x, blockDim.x);
}

}  // namespace
}  // namespace wf
