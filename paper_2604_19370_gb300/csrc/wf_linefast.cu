// Chunked line solves (TMA-staged x pass, column-parallel y pass) and the streaming Kronecker
// matvec.
//
// Paper: Sec. 4 ("Cost of directional implicit solves"): each directional system
// is a set of independent banded 1-D solves (half-bandwidth p) along x or y.
//
// Every line is cut into at most 32 chunks; one thread owns one chunk (`base`
// values, or the last chunk of at most base + 2p values), runs the chunk-local LU
// substitution with the recurrence in registers, solves the p x p interface
// systems of truncated SPIKE with its neighbours' boundary values and applies the
// spike corrections.  LU factors and spikes come from shared memory in their
// compact form: with uniform open knots every interior chunk has the same factors,
// so a CTA stages three chunk types (first, interior, last) whatever the length.
//
// x pass: one warp per row, one lane per chunk.  The rows of a CTA are contiguous
// in memory and move with one TMA bulk copy each way (cp.async.bulk with an
// mbarrier); neighbouring chunks exchange boundary values by warp shuffles.
// y pass: a CTA owns G columns; lanes of neighbouring columns read and write
// contiguous runs of G elements per row, 16 or 32 loads in flight per thread.
#include "wf_internal.h"

#include "wf_line_blocks.cuh"

namespace wf {

namespace {

// x pass.  CTA = G lines; a warp solves 32 / lanes lines, lane k of a line's group owns chunk k
// (C <= lanes per line).
// The G rows are contiguous in memory: one bulk copy stages them, one bulk store writes them back.
// Chunk lengths are odd, so the 32 lanes of a warp read 32 distinct shared-memory banks.
template <typename P, int PD, bool PRE>
__global__ void __launch_bounds__(256) k_xsolve_warp(const FastArgs<P> a) {
    constexpr int W = 2 * PD + 1;
    if (!scene_active(a.b)) return;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const Chunks ch = a.ch;
    const int N = ch.N, C = ch.C, base = ch.base, G = a.G;
    const int mmax = base + 2 * PD;
    const int arr = blockIdx.y;
    const LineView<P> v = scene_line(a, arr);
    const int j0 = blockIdx.x * G;
    const int rows = min(G, a.nlines - j0);
    const size_t row_bytes = (size_t)a.pitch * sizeof(P);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
    constexpr bool pre = PRE;
    const int sp = a.sp;                                           // shared-memory row stride
    P* rowbuf = reinterpret_cast<P*>(smem_raw + 128);             // [G][sp]
    // pre: T* rows j0-p .. j0+G+p-1 at stride tsp, values at column offset HO, zero halo columns
    // on either side so that the column sweep needs no bounds checks
    constexpr int HO = 4;
    const int tsp = a.tsp;
    P* tbuf = rowbuf + (size_t)G * sp;
    const FacSmem<P, PD> fm(tbuf + (pre ? (size_t)(G + 2 * PD) * tsp : 0), mmax);  // factors, then pre: bands
    const P* __restrict__ in = pre ? v.preF : v.in;
    P* out = v.out;
    // rows of the halo block that exist (pre): lo .. hi-1
    const int lo = max(0, j0 - PD), hi = min(a.nlines, j0 + rows + PD);

    // factors: one bulk copy of the operator's padded block beside the rows, else staged element
    // by element
    const bool fbulk = a.tma && v.fpad != nullptr;
    const uint32_t fbytes = (uint32_t)(fac_elems<PD>(mmax) * sizeof(P));
    bool staged = true;
    if (pre) {
        // halo rows outside the domain read as zero; so do the PD columns left of every row
        for (int r = j0 - PD; r < j0 + rows + PD; ++r) {
            P* row = tbuf + (size_t)(r - (j0 - PD)) * tsp;
            if (r >= lo && r < hi) {
                if (tid < PD) row[HO - PD + tid] = P(0);
            } else {
                for (int x = tid; x < tsp; x += blockDim.x) row[x] = P(0);
            }
        }
    }
    if (a.tma) {
        // one bulk copy per row (the shared-memory stride differs from the global pitch);
        // thread 0 arms the barrier with the total, the lanes of warp 0 issue the copies
        if (tid == 0) {
            mbar_init(bar, 1);
            mbar_fence_init();
            const uint32_t bytes = (uint32_t)(rows * row_bytes);
            const uint32_t tbytes = pre ? (uint32_t)((hi - lo) * row_bytes) : 0u;
            mbar_expect_tx(bar, bytes + tbytes + (fbulk ? fbytes : 0u));
        }
        __syncwarp();
        if (warp == 0) {
            if (fbulk && lane == 31) bulk_load(fm.F, v.fpad, fbytes, bar);
            for (int r = lane; r < rows; r += 32)
                bulk_load(rowbuf + (size_t)r * sp, in + (size_t)(j0 + r) * a.pitch, (uint32_t)row_bytes, bar);
            if (pre)
                for (int r = lo + lane; r < hi; r += 32)
                    bulk_load(tbuf + (size_t)(r - (j0 - PD)) * tsp + HO, v.preT + (size_t)r * a.pitch,
                              (uint32_t)row_bytes, bar);
        }
    } else {
        for (int r = 0; r < rows; ++r)
            for (int x = tid; x < N; x += blockDim.x) rowbuf[(size_t)r * sp + x] = in[(size_t)(j0 + r) * a.pitch + x];
        if (pre)
            for (int r = lo; r < hi; ++r)
                for (int x = tid; x < N; x += blockDim.x)
                    tbuf[(size_t)(r - (j0 - PD)) * tsp + HO + x] = v.preT[(size_t)r * a.pitch + x];
    }
    if (!fbulk) stage_factors<P, PD>(v, mmax, fm);
    if (pre) {
        P* bco = fm.end();
        for (int i = tid; i < rows * W; i += blockDim.x) {
            const int r = i / W, d = i - r * W;
            bco[(size_t)r * 2 * W + d] = a.pc1 * v.pB1[(size_t)(j0 + r) * W + d];
            bco[(size_t)r * 2 * W + W + d] = v.pA2 ? a.pc2 * v.pB2[(size_t)(j0 + r) * W + d] : P(0);
        }
    }
    __syncthreads();  // mbarrier initialised, factors staged, halo zeroed
    if (a.tma) staged = mbar_wait_bounded(bar, 0, a.wait_ns);
    staged = __syncthreads_and(staged);  // one decision for the whole CTA (barriers follow)
    if (!staged) {
        // drain the copies in flight before the shared memory is released; the step's output is
        // not valid (bit 4 invalidates it for the whole handle)
        mbar_drain(bar, 0);
        if (tid == 0 && v.tstatus) atomicOr(v.tstatus, 4);
        return;
    }
    if (pre) {
        // the PD columns right of every staged row read as zero (they may hold row padding)
        for (int r = lo; r < hi; ++r)
            if (tid < PD) tbuf[(size_t)(r - (j0 - PD)) * tsp + HO + N + tid] = P(0);
        __syncthreads();
        // R = preFscale F + (pA1 (x) pc1 pB1) T + (pA2 (x) pc2 pB2) T.  Work item = one column and
        // a group of rh output rows: the x bands of the column are loaded once and applied to the
        // rh + 2p staged rows the group needs, whose results pass through a W-row register window
        // that the y bands reduce.  The number of row groups nh balances N * nh items over the
        // CTA's threads against the 2p rows each group re-reads.
        const P* __restrict__ bco = fm.end();  // [G][2][W], scaled by pc1 / pc2
        const int nt = blockDim.x;
        int nh = 1, rh = rows;
        long best;
        {
            best = (long)((N + nt - 1) / nt) * (rows + 2 * PD);
            for (int cand = 2; cand <= 8 && cand <= rows; cand *= 2) {
                const int h = (rows + cand - 1) / cand;
                const long cost = (long)((N * cand + nt - 1) / nt) * (h + 2 * PD);
                if (cost < best) {
                    best = cost;
                    nh = cand;
                    rh = h;
                }
            }
        }
        // alternatively every thread takes an equal run of L (column, row) pairs in column-major
        // order (at most L / rows + 2 column pieces): no ragged last round when N is just above
        // a multiple of the thread count
        const long total = (long)N * rows;
        const long L = (total + nt - 1) / nt;
        const bool flat = L + 2 * PD * (L / rows + 2) < best;
        // rows r0 .. r1-1 of column x
        auto column_run = [&](int x, int r0, int r1) {
            P a1v[W], a2v[W], w1[W], w2[W];
#pragma unroll
            for (int d = 0; d < W; ++d) {
                a1v[d] = v.pA1[(size_t)x * W + d];
                a2v[d] = v.pA2 ? v.pA2[(size_t)x * W + d] : P(0);
                w1[d] = P(0);
                w2[d] = P(0);
            }
            const P* tcol = tbuf + (size_t)r0 * tsp + HO - PD + x;
            P* rcol = rowbuf + (size_t)r0 * sp + x;
            for (int r = r0; r < r1 + 2 * PD; ++r) {
                P t1 = 0, t2 = 0;
#pragma unroll
                for (int dk = 0; dk < W; ++dk) {
                    const P val = tcol[dk];
                    t1 += a1v[dk] * val;
                    t2 += a2v[dk] * val;
                }
                tcol += tsp;
#pragma unroll
                for (int d = 0; d + 1 < W; ++d) {
                    w1[d] = w1[d + 1];
                    w2[d] = w2[d + 1];
                }
                w1[W - 1] = t1;
                w2[W - 1] = t2;
                if (r >= r0 + 2 * PD) {
                    const P* bj = bco + (size_t)(r - 2 * PD) * 2 * W;
                    P acc = a.preFscale * *rcol;
#pragma unroll
                    for (int dl = 0; dl < W; ++dl) acc = fma(bj[dl], w1[dl], fma(bj[W + dl], w2[dl], acc));
                    *rcol = acc;
                    rcol += sp;
                }
            }
        };
        if (flat) {
            long s0 = (long)tid * L;
            const long s1 = min(total, s0 + L);
            while (s0 < s1) {
                const int x = (int)(s0 / rows), r0 = (int)(s0 - (long)x * rows);
                const int r1 = (int)min((long)rows, (long)r0 + (s1 - s0));
                column_run(x, r0, r1);
                s0 += r1 - r0;
            }
        } else {
            for (int item = tid; item < N * nh; item += nt) {
                const int grp = item / N, x = item - grp * N;
                column_run(x, grp * rh, min(rows, grp * rh + rh));
            }
        }
        __syncthreads();
    }

    // lanes per line: 32 >> (5 - lsh); line r of the CTA = warp * lines-per-warp + lane / lanes
    const int k = lane & ((1 << a.lsh) - 1);
    const int r = (warp << (5 - a.lsh)) + (lane >> a.lsh);
    const bool active = r < rows && k < C;
    const int m = (k < C - 1) ? base : ch.last;
    P* g = rowbuf + (size_t)(r < rows ? r : 0) * sp + (size_t)k * base;
    const int t = chunk_type(ch, k < C ? k : 0);
    if (active) {
        lu_forward<P, PD>(g, m, fm.F + t * mmax * FacW<PD>::F);
        lu_backward<P, PD>(g, m, fm.U + t * mmax * FacW<PD>::U);
    }
    __syncwarp();
    P top[PD], bot[PD], nxt_top[PD], prv_bot[PD];
#pragma unroll
    for (int q = 0; q < PD; ++q) {
        top[q] = active ? g[q] : P(0);
        bot[q] = (active && k + 1 < C) ? g[base - PD + q] : P(0);
    }
#pragma unroll
    for (int q = 0; q < PD; ++q) {
        nxt_top[q] = __shfl_down_sync(0xffffffffu, top[q], 1);
        prv_bot[q] = __shfl_up_sync(0xffffffffu, bot[q], 1);
    }
    P tn[PD], bp[PD];
    interface_solve<P, PD>(ch, k < C ? k : 0, mmax, fm.S, fm.E, top, bot, nxt_top, prv_bot, tn, bp);
    if (active) spike_fix<P, PD>(g, m, fm.S + t * mmax * FacW<PD>::S, tn, bp);
    if (a.tma) {
        fence_proxy_async_smem();
        __syncthreads();
        if (warp == 0) {
            bool issued = false;
            for (int r = lane; r < rows; r += 32) {
                bulk_store(out + (size_t)(j0 + r) * a.pitch, rowbuf + (size_t)r * sp, (uint32_t)row_bytes);
                issued = true;
            }
            if (issued) bulk_commit_and_wait_read();
        }
    } else {
        __syncthreads();
        for (int r = 0; r < rows; ++r)
            for (int x = tid; x < N; x += blockDim.x) out[(size_t)(j0 + r) * a.pitch + x] = rowbuf[(size_t)r * sp + x];
    }
}

// y pass.  CTA = G columns x C chunks (blockDim = G*C <= 256); thread tid = k*G + c owns chunk k
// of column c in its private shared-memory strip (odd stride: distinct banks).  The column values
// are loaded 16 or 32 rows at a time and eliminated forward as they arrive, so the strip is written
// once before the backward sweep; the increment base is added on the final store.  Threads of
// columns past the last line solve a copy of the last line and store nothing.
template <typename P, int PD, int B>
__global__ void __launch_bounds__(256) k_ysolve_cols(const FastArgs<P> a) {
    constexpr int W = 2 * PD + 1, B2 = 8;
    constexpr int NF = FacW<PD>::F, NU = FacW<PD>::U, NS = FacW<PD>::S;
    if (!scene_active(a.b)) return;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int tid = threadIdx.x;
    const Chunks ch = a.ch;
    const int N = ch.N, C = ch.C, base = ch.base, G = a.G, mpad = a.mpad;
    const int mmax = base + 2 * PD;
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);  // 16 bytes: the factors' mbarrier
    const FacSmem<P, PD> fm(reinterpret_cast<P*>(smem_raw + 16), mmax);
    P* buf = fm.end();  // [nt][mpad]
    const int arr = blockIdx.y;
    const int k = tid / G, c = tid - k * G;
    const int s = k * base;
    const int m = (k < C - 1) ? base : ch.last;
    const int t = chunk_type(ch, k);
    const int line_raw = blockIdx.x * G + c;
    const bool valid = line_raw < a.nlines;
    const int line = valid ? line_raw : a.nlines - 1;
    const LineView<P> v = scene_line(a, arr);
    const size_t pitch = (size_t)a.pitch;
    P* g = buf + (size_t)tid * mpad;

    // factors: one bulk copy of the operator's padded block (bounded wait; a CTA that gives up
    // stores nothing and sets bit 4 of the slot's flag word), else staged element by element
    const bool fbulk = v.fpad != nullptr;
    if (fbulk) {
        if (tid == 0) {
            const uint32_t fbytes = (uint32_t)(fac_elems<PD>(mmax) * sizeof(P));
            mbar_init(bar, 1);
            mbar_fence_init();
            mbar_expect_tx(bar, fbytes);
            bulk_load(fm.F, v.fpad, fbytes, bar);
        }
    } else {
        stage_factors<P, PD>(v, mmax, fm);
    }
    __syncthreads();
    if (fbulk) {
        const bool ok = __syncthreads_and(mbar_wait_bounded(bar, 0, a.wait_ns));
        if (!ok) {
            mbar_drain(bar, 0);
            if (tid == 0 && v.tstatus) atomicOr(v.tstatus, 4);
            return;
        }
    }
    const P* __restrict__ pre = v.premul;
    const P* Fk = fm.F + t * mmax * NF;
    P prev[PD];
#pragma unroll
    for (int i = 0; i < PD; ++i) prev[i] = P(0);
    if (pre) {
        // right-hand side prescale (premul band (x) I) in: rows s .. s+m-1 of the product
        const P ps = v.prescale;
        for (int o = 0; o < m; ++o) {
            const int row = s + o;
            P acc = 0;
#pragma unroll
            for (int d = 0; d < W; ++d) {
                const int rr = row + d - PD;
                if (rr >= 0 && rr < N) acc += pre[(size_t)row * W + d] * v.in[(size_t)rr * pitch + line];
            }
            P x[1] = {ps * acc};
            fwd_rows<P, PD, 1>(x, Fk + o * NF, prev);
            g[o] = x[0];
        }
    } else {
        const P* __restrict__ src = v.in + (size_t)s * pitch + line;
        int o = 0;
        for (; o + B <= m; o += B) {
            P r[B];
#pragma unroll
            for (int q = 0; q < B; ++q) r[q] = src[q * pitch];
            src += B * pitch;
            fwd_rows<P, PD, B>(r, Fk + o * NF, prev);
#pragma unroll
            for (int q = 0; q < B; ++q) g[o + q] = r[q];
        }
        for (; o < m; ++o) {
            P r[1] = {*src};
            src += pitch;
            fwd_rows<P, PD, 1>(r, Fk + o * NF, prev);
            g[o] = r[0];
        }
    }
    lu_backward<P, PD>(g, m, fm.U + t * mmax * NU);
    __syncthreads();
    const P* gn = buf + (size_t)((k + 1 < C ? k + 1 : k) * G + c) * mpad;
    const P* gp = buf + (size_t)((k > 0 ? k - 1 : k) * G + c) * mpad + (base - PD);
    P tn[PD], bp[PD];
    interface_solve<P, PD>(ch, k, mmax, fm.S, fm.E, g, g + (base - PD), gn, gp, tn, bp);
    if (!valid) return;  // no barrier follows
    const P* Sk = fm.S + t * mmax * NS;
    const P* __restrict__ bs = v.base ? v.base + (size_t)s * pitch + line : nullptr;
    P* dst = v.out + (size_t)s * pitch + line;
    const P tmax = a.tmax;
    bool bad = false;
    // final rows: spike correction, increment base, store, guard
    auto finish = [&](auto nrows, int o) {
        constexpr int R = decltype(nrows)::value;
        P x[R], bv[R];
#pragma unroll
        for (int q = 0; q < R; ++q) {
            x[q] = g[o + q];
            bv[q] = bs ? bs[(size_t)q * pitch] : P(0);
        }
        spike_rows<P, PD, R>(x, Sk + o * NS, tn, bp);
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const P y = x[q] + bv[q];
            dst[(size_t)q * pitch] = y;
            bad |= !(fabs(y) <= tmax);  // also catches NaN
        }
        if (bs) bs += R * pitch;
        dst += R * pitch;
    };
    int o = 0;
    for (; o + B2 <= m; o += B2) finish(std::integral_constant<int, B2>{}, o);
    for (; o < m; ++o) finish(std::integral_constant<int, 1>{}, o);
    if (bad && v.status != nullptr && arr == 0) atomicOr(v.status, 1);
}

// y pass for long lines (many chunks): CTA = 32 columns x C chunks (up to 1024 threads), thread
// tid = k*32 + c owns chunk k of column c, so a warp's loads and stores cover 32 consecutive columns
// (128-byte row pieces) whatever the chunk count.  The chunk's partial results are kept in the
// pass's input array (the right-hand side, dead after the pass: LineArgs::in_dead) instead of a
// shared-memory strip (a strip per thread of a long chunk fills the shared memory with one CTA of
// eight columns): each thread overwrites the input elements it has read and reads them back in the
// later sweeps (its own writes, in program order; the CTA's column block stays in L2); neighbouring
// chunks exchange their first and last p values through shared memory.
// Per column the operations, and their order, are those of k_ysolve_cols: the same bits.
template <typename P, int PD, int B>
__global__ void __launch_bounds__(1024) k_ysolve_long(const FastArgs<P> a) {
    constexpr int B2 = 8;
    constexpr int NF = FacW<PD>::F, NU = FacW<PD>::U, NS = FacW<PD>::S;
    if (!scene_active(a.b)) return;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int tid = threadIdx.x;
    const Chunks ch = a.ch;
    const int C = ch.C, base = ch.base;
    constexpr int G = 32;
    const int mmax = base + 2 * PD;
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);  // 16 bytes: the factors' mbarrier
    const FacSmem<P, PD> fm(reinterpret_cast<P*>(smem_raw + 16), mmax);
    P* xch = fm.end();  // [C][G][2p]: the first and the last p values of every chunk
    const int arr = blockIdx.y;
    const int k = tid / G, c = tid - k * G;
    const int s = k * base;
    const int m = (k < C - 1) ? base : ch.last;
    const int t = chunk_type(ch, k);
    const int line = blockIdx.x * G + c;
    const bool valid = line < a.nlines;  // threads past the last line only take part in the barriers
    const LineView<P> v = scene_line(a, arr);
    const size_t pitch = (size_t)a.pitch;
    const bool fbulk = v.fpad != nullptr;
    if (fbulk) {
        if (tid == 0) {
            const uint32_t fbytes = (uint32_t)(fac_elems<PD>(mmax) * sizeof(P));
            mbar_init(bar, 1);
            mbar_fence_init();
            mbar_expect_tx(bar, fbytes);
            bulk_load(fm.F, v.fpad, fbytes, bar);
        }
    } else {
        stage_factors<P, PD>(v, mmax, fm);
    }
    __syncthreads();
    if (fbulk) {
        const bool ok = __syncthreads_and(mbar_wait_bounded(bar, 0, a.wait_ns));
        if (!ok) {
            mbar_drain(bar, 0);
            if (tid == 0 && v.tstatus) atomicOr(v.tstatus, 4);
            return;
        }
    }
    P* g = const_cast<P*>(v.in) + (size_t)s * pitch + (valid ? line : 0);  // this chunk's input elements
    P top[PD], bot[PD];
    if (valid) {
        const P* Fk = fm.F + t * mmax * NF;
        P prev[PD];
#pragma unroll
        for (int i = 0; i < PD; ++i) prev[i] = P(0);
        const P* src = v.in + (size_t)s * pitch + line;  // the elements g overwrites, each after its read
        int o = 0;
        for (; o + B <= m; o += B) {
            P r[B];
#pragma unroll
            for (int q = 0; q < B; ++q) r[q] = src[q * pitch];
            src += B * pitch;
            fwd_rows<P, PD, B>(r, Fk + o * NF, prev);
#pragma unroll
            for (int q = 0; q < B; ++q) g[(size_t)(o + q) * pitch] = r[q];
        }
        for (; o < m; ++o) {
            P r[1] = {*src};
            src += pitch;
            fwd_rows<P, PD, 1>(r, Fk + o * NF, prev);
            g[(size_t)o * pitch] = r[0];
        }
        // backward substitution from the last row up, on the elements just written
        const P* Uk = fm.U + t * mmax * NU;
#pragma unroll
        for (int i = 0; i < PD; ++i) prev[i] = P(0);
        int top_r = m - 1;
        for (; top_r - B2 + 1 >= 0; top_r -= B2) {
            P gv[B2];
#pragma unroll
            for (int q = 0; q < B2; ++q) gv[q] = g[(size_t)(top_r - q) * pitch];
            bwd_rows<P, PD, B2>(gv, Uk + top_r * NU, prev);
#pragma unroll
            for (int q = 0; q < B2; ++q) g[(size_t)(top_r - q) * pitch] = gv[q];
        }
        for (; top_r >= 0; --top_r) {
            P gv[1] = {g[(size_t)top_r * pitch]};
            bwd_rows<P, PD, 1>(gv, Uk + top_r * NU, prev);
            g[(size_t)top_r * pitch] = gv[0];
        }
        P* mine = xch + (size_t)tid * 2 * PD;
#pragma unroll
        for (int q = 0; q < PD; ++q) {
            top[q] = g[(size_t)q * pitch];
            // the last chunk may be shorter than base (its last p values are not used)
            bot[q] = (k + 1 < C) ? g[(size_t)(base - PD + q) * pitch] : P(0);
            mine[q] = top[q];
            mine[PD + q] = bot[q];
        }
    }
    __syncthreads();
    if (!valid) return;  // no barrier follows
    const P* nx = xch + (size_t)((k + 1 < C ? k + 1 : k) * G + c) * 2 * PD;
    const P* pv = xch + (size_t)((k > 0 ? k - 1 : k) * G + c) * 2 * PD + PD;
    P nt[PD], pb[PD], tn[PD], bp[PD];
#pragma unroll
    for (int q = 0; q < PD; ++q) {
        nt[q] = nx[q];
        pb[q] = pv[q];
    }
    interface_solve<P, PD>(ch, k, mmax, fm.S, fm.E, top, bot, nt, pb, tn, bp);
    const P* Sk = fm.S + t * mmax * NS;
    const P* bs = v.base ? v.base + (size_t)s * pitch + line : nullptr;  // may be the output array
    P* dst = v.out + (size_t)s * pitch + line;
    const P tmax = a.tmax;
    bool bad = false;
    auto finish = [&](auto nrows, int o) {
        constexpr int R = decltype(nrows)::value;
        P x[R], bv[R];
#pragma unroll
        for (int q = 0; q < R; ++q) {
            x[q] = g[(size_t)(o + q) * pitch];
            bv[q] = bs ? bs[(size_t)(o + q) * pitch] : P(0);
        }
        spike_rows<P, PD, R>(x, Sk + o * NS, tn, bp);
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const P y = x[q] + bv[q];
            dst[(size_t)(o + q) * pitch] = y;
            bad |= !(fabs(y) <= tmax);  // also catches NaN
        }
    };
    int o = 0;
    for (; o + B2 <= m; o += B2) finish(std::integral_constant<int, B2>{}, o);
    for (; o < m; ++o) finish(std::integral_constant<int, 1>{}, o);
    if (bad && v.status != nullptr && arr == 0) atomicOr(v.status, 1);
}

template <typename P, int PD, bool X>
cudaError_t run_fast(const LineArgs& a, cudaStream_t s) {
    constexpr int W = 2 * PD + 1;
    const Chunks& ch = a.f[0].ch;
    if (ch.C > 32) return cudaErrorNotSupported;
    const int mmax = ch.base + 2 * PD;
    const size_t fbytes = (size_t)fac_elems<PD>(mmax) * sizeof(P);
    FastArgs<P> f;
    f.nlines = a.nlines;
    f.pitch = a.pitch;
    f.ch = ch;
    for (int q = 0; q < 2; ++q) {
        f.in[q] = (const P*)a.in[q];
        f.out[q] = (P*)a.out[q];
        f.base[q] = (const P*)a.base[q];
        f.premul[q] = (const P*)a.premul[q];
        f.prescale[q] = (P)a.prescale[q];
        f.luc[q] = (const P*)a.f[q].luc;
        f.spkc[q] = (const P*)a.f[q].spkc;
        f.Ec[q] = (const P*)a.f[q].Ec;
        f.fpad[q] = (const P*)a.f[q].fpad;
    }
    f.status = a.status;
    f.tstatus = a.tstatus;
    f.wait_ns = a.wait_ns;
    f.tmax = (P)a.tmax;
    f.b = a.b;
    f.mpad = (ch.base > ch.last ? ch.base : ch.last) | 1;
    f.preT = (const P*)a.preT;
    f.preF = (const P*)a.preF;
    f.preFscale = (P)a.preFscale;
    f.pc1 = (P)a.pc1;
    f.pc2 = (P)a.pc2;
    f.pA1 = (const P*)a.pA1;
    f.pB1 = (const P*)a.pB1;
    f.pA2 = (const P*)a.pA2;
    f.pB2 = (const P*)a.pB2;
    if (!X && a.preT) return cudaErrorNotSupported;
    if (X) {
        // rows per CTA: as many warps as fit 100 KB of staged rows (at least one)
        const size_t row_bytes = (size_t)a.pitch * sizeof(P);
        const bool pre = a.preT != nullptr;
        if (pre && a.narr != 1) return cudaErrorNotSupported;
        // lines per warp: as many as the chunks allow (C <= 8: four, C <= 16: two), or fewer
        int lsh = ch.C <= 8 ? 3 : (ch.C <= 16 ? 4 : 5);
        if (a.rpw == 1) lsh = 5;
        else if (a.rpw == 2 && lsh < 4) lsh = 4;
        const int lpw = 1 << (5 - lsh);
        // shared-memory row stride: the lines of a warp start L banks apart (L = lanes per line,
        // chunk lengths odd), so its lanes hit distinct banks; 16-byte multiple for bulk copies
        const int L = 32 >> (5 - lsh);
        const int slots = sizeof(P) == 4 ? 32 : 16;  // bank-width words per wavefront
        int sp = a.pitch;
        if (L < slots)
            while (sp % (2 * L) != L || (sp * sizeof(P)) % 16 != 0) ++sp;
        const size_t srow = (size_t)sp * sizeof(P);
        const int tsp = pre ? round4(4 + a.pitch + PD) : 0;  // staged T* rows: 4 left, PD right halo
        const size_t trow = (size_t)tsp * sizeof(P);
        auto need = [&](int g) {
            return 128 + g * srow + (pre ? (g + 2 * PD) * trow + (size_t)g * 2 * W * sizeof(P) : 0) + fbytes;
        };
        // lines per CTA: up to 8 warps' worth, fewer when the staged rows need more than 100 KB
        int G = 8 * lpw;
        if (a.G > 0 && a.G < G) G = a.G < lpw ? lpw : a.G;
        G = (G + lpw - 1) / lpw * lpw;
        while (G > lpw && need(G) > 100 * 1024) G = ((G / 2) + lpw - 1) / lpw * lpw;
        const size_t smem = need(G);
        if (smem > 227 * 1024) return cudaErrorNotSupported;
        bool aligned = (row_bytes % 16 == 0) && (a.b.sbytes % 16 == 0);
        for (int q = 0; q < a.narr; ++q)
            aligned = aligned && ((uintptr_t)(pre ? a.preF : a.in[q]) % 16 == 0) && ((uintptr_t)a.out[q] % 16 == 0);
        if (pre) aligned = aligned && ((uintptr_t)a.preT % 16 == 0);
        f.G = G;
        f.lsh = lsh;
        f.sp = sp;
        f.tsp = tsp;
        f.tma = aligned ? 1 : 0;
        auto kern = pre ? k_xsolve_warp<P, PD, true> : k_xsolve_warp<P, PD, false>;
        cudaError_t e = allow_dynamic_smem(kern, (size_t)smem);
        if (e != cudaSuccess) return e;
        dim3 grid((a.nlines + G - 1) / G, a.narr, a.b.S);
        kern<<<grid, 32 * (G / lpw), smem, s>>>(f);
        count_launches(1);
    } else {
        int sms = 152, dev = 0;
        if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        // long lines (more than 8 chunks) whose input is dead after the pass, no prescale band, and
        // enough 32-column blocks for half the SMs: 32 columns per CTA, partial results in the input
        bool lng = a.in_dead && ch.C > 8 && (long)((a.nlines + 31) / 32) * a.narr * a.b.S >= sms / 2;
        for (int q = 0; q < a.narr; ++q) lng = lng && a.premul[q] == nullptr;
        if (lng) {
            const int ntl = 32 * ch.C;
            const size_t smeml = 16 + fbytes + (size_t)ntl * 2 * PD * sizeof(P);
            f.G = 32;
            f.tma = 0;
            dim3 grid((a.nlines + 31) / 32, a.narr, a.b.S);
            auto kern = k_ysolve_long<P, PD, 16>;
            cudaError_t e = allow_dynamic_smem(kern, smeml);
            if (e != cudaSuccess) return e;
            kern<<<grid, ntl, smeml, s>>>(f);
            count_launches(1);
            return cudaGetLastError();
        }
        int G = a.G > 0 ? (a.G < 256 ? a.G : 256) : (sizeof(P) == 4 ? 8 : 4);
        while (G > 1 && G * ch.C > 256) G /= 2;
        const int nt = G * ch.C;
        if (nt > 256) return cudaErrorNotSupported;
        const size_t smem = 16 + fbytes + (size_t)nt * f.mpad * sizeof(P);
        if (smem > 227 * 1024) return cudaErrorNotSupported;
        f.G = G;
        f.tma = 0;
        // rows loaded per batch: 32 when the launch leaves at most two CTAs per SM (its threads then
        // wait on load latency, and more loads in flight pay), else 16 (fewer registers, more CTAs)
        dim3 grid((a.nlines + G - 1) / G, a.narr, a.b.S);
        const bool wide = (long)grid.x * grid.y * grid.z <= 2L * sms;
        auto kern = wide ? k_ysolve_cols<P, PD, 32> : k_ysolve_cols<P, PD, 16>;
        cudaError_t e = allow_dynamic_smem(kern, (size_t)smem);
        if (e != cudaSuccess) return e;
        kern<<<grid, nt, smem, s>>>(f);
        count_launches(1);
    }
    return cudaGetLastError();
}

// Padded factor block of one operator: the layout stage_factors builds in shared memory, written
// once to global memory when the operator is factored (padding entries zero).
template <typename P, int PD>
__global__ void k_pad_factors(const P* __restrict__ luc, const P* __restrict__ spkc, const P* __restrict__ Ec,
                              int mmax, P* out) {
    const FacSmem<P, PD> fm(out, mmax);
    fill_factors<P, PD>(luc, spkc, Ec, mmax, fm, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

// ---- streaming explicit Kronecker matvec ---------------------------------------------
// R = Fscale F + c1 (A1^x (x) B1^y) T + c2 (A2^x (x) B2^y) T.  A warp owns 32 columns (lane L
// <-> column X0 - p + L; lanes p .. 31-p are outputs) and RS output rows: it issues every load
// of its RS + 2p rows of T and RS rows of F first, x-convolves each row with neighbours'
// values taken by shuffles, and reduces the y bands from registers.  No shared memory, no
// barriers, every warp independent.  Values outside the domain are zeros, and the operations
// (and their order) are those of the right-hand side fused into the x pass.
template <typename P, int PD, int RS>
__global__ void __launch_bounds__(128) k_matvec_stream(int Nx, int Ny, int pitch, const P* __restrict__ T,
                                                       const P* __restrict__ F, P* R, const P* __restrict__ A1,
                                                       const P* __restrict__ B1, const P* __restrict__ A2,
                                                       const P* __restrict__ B2, P Fscale, P c1, P c2, Batch b,
                                                       int nstrips, int nsegs) {
    constexpr int W = 2 * PD + 1, NR = RS + 2 * PD;
    if (!scene_active(b)) return;
    const int lane = threadIdx.x & 31;
    const int item = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (item >= nstrips * nsegs) return;  // whole warp
    T = scene_ptr(T, b);
    F = scene_ptr(F, b);
    R = scene_ptr(R, b);
    A1 = scene_ptr(A1, b);
    B1 = scene_ptr(B1, b);
    A2 = scene_ptr(A2, b);
    B2 = scene_ptr(B2, b);
    const int sg = item / nstrips, st = item - sg * nstrips;
    const int x = st * (32 - 2 * PD) - PD + lane;  // this lane's column
    const bool xok = x >= 0 && x < Nx;
    const bool out = lane >= PD && lane < 32 - PD && x < Nx;
    const int j0 = sg * RS;  // first output row
    // interior segment: every T row it reads exists and every output row has the interior
    // y bands (rows 2p .. Ny-2p-1 of a band all equal row 2p), so no row needs a guard
    const bool yint = j0 >= 2 * PD && j0 + RS + 2 * PD <= Ny;
    P tv[NR], fv[RS];
    if (yint) {
        const P* tp = T + (size_t)(j0 - PD) * pitch + (xok ? x : 0);
        const P* fp = F + (size_t)j0 * pitch + (xok ? x : 0);
#pragma unroll
        for (int i = 0; i < NR; ++i) tv[i] = xok ? tp[(size_t)i * pitch] : P(0);
#pragma unroll
        for (int i = 0; i < RS; ++i) fv[i] = out ? fp[(size_t)i * pitch] : P(0);
    } else {
#pragma unroll
        for (int i = 0; i < NR; ++i) {
            const int r = j0 - PD + i;
            tv[i] = (xok && r >= 0 && r < Ny) ? T[(size_t)r * pitch + x] : P(0);
        }
#pragma unroll
        for (int i = 0; i < RS; ++i) {
            const int r = j0 + i;
            fv[i] = (out && r < Ny) ? F[(size_t)r * pitch + x] : P(0);
        }
    }
    P a1v[W], a2v[W];
#pragma unroll
    for (int d = 0; d < W; ++d) {
        a1v[d] = out ? A1[(size_t)x * W + d] : P(0);
        a2v[d] = (out && A2) ? A2[(size_t)x * W + d] : P(0);
    }
    // x-convolution of every row (outputs lanes read lanes lane - p .. lane + p)
    P w1[NR], w2[NR];
    if constexpr (sizeof(P) == 4 && NR % 2 == 0) {
        // FP32: rows i and i+1 side by side in packed FMAs (per row the same operations)
        float2 a1p[W], a2p[W];
#pragma unroll
        for (int d = 0; d < W; ++d) {
            a1p[d] = make_float2(a1v[d], a1v[d]);
            a2p[d] = make_float2(a2v[d], a2v[d]);
        }
#pragma unroll
        for (int i = 0; i < NR; i += 2) {
            float2 t1 = make_float2(0.f, 0.f), t2 = make_float2(0.f, 0.f);
#pragma unroll
            for (int dk = 0; dk < W; ++dk) {
                const int src = (lane - PD + dk) & 31;
                const float2 val = (dk == PD) ? make_float2(tv[i], tv[i + 1])
                                              : make_float2(__shfl_sync(0xffffffffu, tv[i], src),
                                                            __shfl_sync(0xffffffffu, tv[i + 1], src));
                t1 = __ffma2_rn(a1p[dk], val, t1);
                t2 = __ffma2_rn(a2p[dk], val, t2);
            }
            w1[i] = t1.x;
            w1[i + 1] = t1.y;
            w2[i] = t2.x;
            w2[i + 1] = t2.y;
        }
    } else {
#pragma unroll
        for (int i = 0; i < NR; ++i) {
            P t1 = 0, t2 = 0;
#pragma unroll
            for (int dk = 0; dk < W; ++dk) {
                const P val = (dk == PD) ? tv[i] : __shfl_sync(0xffffffffu, tv[i], (lane - PD + dk) & 31);
                t1 += a1v[dk] * val;
                t2 += a2v[dk] * val;
            }
            w1[i] = t1;
            w2[i] = t2;
        }
    }
    if (!out) return;
    // the interior y bands (rows 2p .. Ny-2p-1 of a band all equal row 2p), where such rows exist
    const bool has_int = Ny > 4 * PD;
    P b1i[W], b2i[W];
#pragma unroll
    for (int d = 0; d < W; ++d) {
        b1i[d] = has_int ? c1 * B1[(size_t)(2 * PD) * W + d] : P(0);
        b2i[d] = (has_int && A2) ? c2 * B2[(size_t)(2 * PD) * W + d] : P(0);
    }
    if (yint) {
        P* rp = R + (size_t)j0 * pitch + x;
#pragma unroll
        for (int o = 0; o < RS; ++o) {
            P acc = Fscale * fv[o];
#pragma unroll
            for (int dl = 0; dl < W; ++dl) acc = fma(b1i[dl], w1[o + dl], fma(b2i[dl], w2[o + dl], acc));
            rp[(size_t)o * pitch] = acc;
        }
        return;
    }
#pragma unroll
    for (int o = 0; o < RS; ++o) {
        const int j = j0 + o;
        if (j >= Ny) break;
        P acc = Fscale * fv[o];
        if (j < 2 * PD || j >= Ny - 2 * PD) {
            // the first and last 2p rows have bands of their own
#pragma unroll
            for (int dl = 0; dl < W; ++dl) {
                const P b1 = c1 * B1[(size_t)j * W + dl];
                const P b2 = A2 ? c2 * B2[(size_t)j * W + dl] : P(0);
                acc = fma(b1, w1[o + dl], fma(b2, w2[o + dl], acc));
            }
        } else {
#pragma unroll
            for (int dl = 0; dl < W; ++dl) acc = fma(b1i[dl], w1[o + dl], fma(b2i[dl], w2[o + dl], acc));
        }
        R[(size_t)j * pitch + x] = acc;
    }
}

}  // namespace

cudaError_t launch_line_fast(int prec, int p, bool xdir, const LineArgs& a, cudaStream_t s) {
    for (int q = 0; q < a.narr; ++q)
        if (!a.f[q].compact || a.f[q].ch.base != a.f[0].ch.base || a.f[q].ch.C != a.f[0].ch.C)
            return cudaErrorNotSupported;
#define WF_FAST(P, PD) return xdir ? run_fast<P, PD, true>(a, s) : run_fast<P, PD, false>(a, s)
    if (prec == 0) {
        switch (p) {
            case 1: WF_FAST(float, 1);
            case 2: WF_FAST(float, 2);
            case 3: WF_FAST(float, 3);
        }
    } else {
        switch (p) {
            case 1: WF_FAST(double, 1);
            case 2: WF_FAST(double, 2);
            case 3: WF_FAST(double, 3);
        }
    }
#undef WF_FAST
    return cudaErrorNotSupported;
}

size_t fac_pad_elems(int p, int mmax) {
    switch (p) {
        case 1: return (size_t)fac_elems<1>(mmax);
        case 2: return (size_t)fac_elems<2>(mmax);
        case 3: return (size_t)fac_elems<3>(mmax);
    }
    return 0;
}

cudaError_t launch_pad_factors(int prec, int p, int mmax, const void* luc, const void* spkc, const void* Ec,
                               void* fpad, cudaStream_t s) {
    const size_t es = prec == 0 ? sizeof(float) : sizeof(double);
    const size_t n = fac_pad_elems(p, mmax);
    if (n == 0) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(fpad, 0, n * es, s);
    if (e != cudaSuccess) return e;
#define WF_PAD(P, PD) \
    k_pad_factors<P, PD><<<4, 256, 0, s>>>((const P*)luc, (const P*)spkc, (const P*)Ec, mmax, (P*)fpad)
    if (prec == 0) {
        switch (p) {
            case 1: WF_PAD(float, 1); break;
            case 2: WF_PAD(float, 2); break;
            case 3: WF_PAD(float, 3); break;
        }
    } else {
        switch (p) {
            case 1: WF_PAD(double, 1); break;
            case 2: WF_PAD(double, 2); break;
            case 3: WF_PAD(double, 3); break;
        }
    }
#undef WF_PAD
    return cudaGetLastError();
}

cudaError_t launch_matvec(int prec, int p, const MatvecArgs& a, cudaStream_t s) {
    // output rows per warp item: 16 (the 2p halo rows and the item's setup spread over more
    // outputs), except 8 for FP64 with p <= 2, where 16 rows would take twice the registers
    constexpr int WARPS = 4;
    if (p < 1 || p > 3) return cudaErrorInvalidValue;
    const int rs = (prec != 0 && p <= 2) ? 8 : 16;
    const int nstrips = (a.Nx + (32 - 2 * p) - 1) / (32 - 2 * p), nsegs = (a.Ny + rs - 1) / rs;
    const long items = (long)nstrips * nsegs;
    dim3 grid((unsigned)((items + WARPS - 1) / WARPS), 1, a.b.S), block(32 * WARPS);
#define WF_MV(P, PD)                                                                                          \
    k_matvec_stream<P, PD, (sizeof(P) == 8 && PD <= 2 ? 8 : 16)><<<grid, block, 0, s>>>(                                         \
        a.Nx, a.Ny, a.pitch, (const P*)a.T, (const P*)a.F, (P*)a.R, (const P*)a.A1, (const P*)a.B1,           \
        (const P*)a.A2, (const P*)a.B2, (P)a.Fscale, (P)a.c1, (P)a.c2, a.b, nstrips, nsegs)
    if (prec == 0) {
        switch (p) {
            case 1: WF_MV(float, 1); break;
            case 2: WF_MV(float, 2); break;
            case 3: WF_MV(float, 3); break;
        }
    } else {
        switch (p) {
            case 1: WF_MV(double, 1); break;
            case 2: WF_MV(double, 2); break;
            case 3: WF_MV(double, 3); break;
        }
    }
#undef WF_MV
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace wf
