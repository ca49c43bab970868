// Persistent line passes: after the quadrature launch of a Peaceman-Rachford step (one F per
// step), one launch runs the rest of the step for every active slot of a batch handle.
//
// Paper: Sec. 3.1 Eq. matrixPR (the two substeps), Sec. 4 (every directional solve is a set
// of independent 1-D line solves, which is what lets one launch cover every pass of a whole
// batch).
//
// After the quadrature (F, Phi and the substep-1 right-hand side R of every slot), the step of
// one slot is five passes, each a set of independent tiles:
//   X1  x lines of R with X_+ and of Phi with M^x, in groups of rows
//   Y1  y lines (R -> T*, Phi -> phi^{n+1}, increment bases added), in groups of columns
//   MV  substep-2 right-hand side R = theta F + (A_x (x) M^y) T* + (M^x (x) A_y) T*, eight warp
//       tiles per item
//   X2  x lines of R with M^x, in groups of rows
//   Y2  y lines with Y_+ (R -> T^{n+1}, base T*), guard, in groups of columns
// The arithmetic of every tile is that of the per-pass kernels (the same device functions or
// the same operations in the same order), so both step forms give the same bits.
//
// Work items (pass, slot, tile) are listed by the host in a wavefront over groups of slots: at
// "time" t the list holds X1 of group t, Y1 of group t-1, ..., Y2 of group t-4, so the fields of
// about five groups are live at once (sized to stay in the L2 cache: a slot's intermediate
// fields go from one pass to the next through L2, not HBM), and consecutive items are
// independent.  A CTA claims the next item from a ticket counter (the next ticket is fetched
// while the current item runs) and, before touching its inputs, waits for the arrival counters
// of the tiles it reads:
//   Y1 columns  <- every X1 row group of its array
//   MV strip    <- the Y1 column groups that cover its columns and halo
//   X2 rows     <- the MV segments that cover them (every strip)
//   Y2 columns  <- every X2 row group
// A tile waits only for tiles with smaller tickets, which are running or done when it is
// claimed, so the launch always makes progress whatever the number of resident CTAs.
// Producers release (stores, barrier, fence, counter add); consumers acquire (ld.acquire on
// the counter, barrier) and read data produced in this launch through L2 (ld.global.cg),
// never through the read-only path.  Every wait is bounded by the handle's wait limit (the
// SM's global timer); a wait that gives up sets the slot's timeout bit and the launch-wide
// abort flag, after which every remaining item is skipped, so a failure costs one limit.
#include <string.h>

#include <algorithm>

#include "wf.h"
#include "wf_line_blocks.cuh"

namespace wf {

namespace {

constexpr int kPT = 256;  // threads per CTA

enum { PH_X1 = 0, PH_Y1 = 1, PH_MV = 2, PH_X2 = 3, PH_Y2 = 4, PH_N = 5 };

// Offsets (ints) of one slot's arrival counters.
struct CntLayout {
    int x1, y1col, mvseg, x2, done, stride;
};

template <typename P>
struct PersistArgs {
    FastArgs<P> x1, y1, x2, y2;
    // substep-2 right-hand side
    const P* mT;
    const P* mF;
    P* mR;
    const P *mA1, *mB1, *mA2, *mB2;
    P mFscale, mc1, mc2;
    int mv_nstrips, mv_nsegs;
    long long sbytes;
    int Nx, Ny, pitch;
    int nxg, nyg;  // row groups of the x passes, column groups of the y passes
    int vec;       // rows 16-byte aligned: stage x lines with 16-byte loads
    const int4* items;
    const int* nitems;
    int* ctl;  // [0] ticket, [1] abort flag, [2] items, [3] items per slot
    int* cnt;  // slot z's counters at cnt + z * cl.stride
    CntLayout cl;
    long long wait_ns;
    int* status;  // slot 0's flag word (slot z: z * sbytes further)
    const int* active;  // per-slot activity flags: an inactive slot's items are skipped
    int* budget;        // per-slot step budgets (NULL: none); a spent one (0) skips the slot too
};

template <typename T>
__device__ __forceinline__ T* shift(T* p, long long off) {
    return p ? reinterpret_cast<T*>(reinterpret_cast<char*>(const_cast<typename std::remove_const<T>::type*>(p)) + off)
             : p;
}

template <typename P>
__device__ __forceinline__ LineView<P> line_at(const FastArgs<P>& a, int arr, long long off) {
    const bool one = arr != 0;
    LineView<P> v;
    v.in = shift(one ? a.in[1] : a.in[0], off);
    v.out = shift(one ? a.out[1] : a.out[0], off);
    v.base = shift(one ? a.base[1] : a.base[0], off);
    v.premul = nullptr;
    v.prescale = P(0);
    v.luc = shift(one ? a.luc[1] : a.luc[0], off);
    v.spkc = shift(one ? a.spkc[1] : a.spkc[0], off);
    v.Ec = shift(one ? a.Ec[1] : a.Ec[0], off);
    v.fpad = nullptr;
    v.status = shift(a.status, off);
    v.tstatus = nullptr;
    v.preT = v.preF = v.pA1 = v.pB1 = v.pA2 = v.pB2 = nullptr;
    return v;
}

__device__ __forceinline__ int ld_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_relaxed(const int* p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long gtime() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait until *c >= target.  false: the wait gave up (limit reached: the slot's timeout bit and
// the abort flag are set) or another wait already did (abort flag seen).  Limit 0 gives up at
// once without looking, so that tests can take this path deterministically.
template <typename P>
__device__ bool wait_count(const PersistArgs<P>& A, const int* c, int target, int* slot_status) {
    if (A.wait_ns > 0) {
        if (ld_acquire(c) >= target) return true;
        const unsigned long long t0 = gtime();
        for (unsigned it = 1;; ++it) {
            if (ld_acquire(c) >= target) return true;
            if (ld_relaxed(A.ctl + 1)) return false;
            if ((it & 7u) == 0u && (long long)(gtime() - t0) > A.wait_ns) break;
            __nanosleep(64);
        }
    }
    atomicExch(A.ctl + 1, 1);
    if (slot_status) atomicOr(slot_status, WF_STATUS_TIMEOUT);
    return false;
}

__device__ __forceinline__ void arrive(int* c) {
    __threadfence();
    atomicAdd(c, 1);
}

// ---- x-line tile (whole CTA): G lines of one array -----------------------------------------
// The operations of k_xsolve_warp (without the fused right-hand side); rows are staged from L2
// with plain loads (they were written by other CTAs of this launch).  `restage`: the factors in
// shared memory are not those of this (slot, operator).
template <typename P, int PD>
__device__ void x_tile(const PersistArgs<P>& A, const FastArgs<P>& a, int z, int arr, int j0, unsigned char* smem,
                       bool restage, int tid, int nt) {
    const int warp = tid >> 5, lane = tid & 31;
    const Chunks ch = a.ch;
    const int N = ch.N, C = ch.C, base = ch.base, G = a.G;
    const int mmax = base + 2 * PD;
    const long long off = (long long)z * A.sbytes;
    const LineView<P> v = line_at(a, arr, off);
    const int rows = min(G, a.nlines - j0);
    const int sp = a.sp;
    const size_t pitch = (size_t)a.pitch;
    P* rowbuf = reinterpret_cast<P*>(smem);
    const FacSmem<P, PD> fm(rowbuf + (size_t)G * sp, mmax);
    if (sizeof(P) == 4 && A.vec) {
        const int n4 = (N + 3) >> 2;  // the row padding beyond N is copied through unchanged
        for (int i = tid; i < rows * n4; i += nt) {
            const int r = i / n4, c = i - r * n4;
            const float4 val = __ldcg(reinterpret_cast<const float4*>(v.in + (size_t)(j0 + r) * pitch) + c);
            *reinterpret_cast<float4*>(rowbuf + (size_t)r * sp + 4 * c) = val;
        }
    } else {
        for (int i = tid; i < rows * N; i += nt) {
            const int r = i / N, x = i - r * N;
            rowbuf[(size_t)r * sp + x] = __ldcg(v.in + (size_t)(j0 + r) * pitch + x);
        }
    }
    if (restage) stage_factors<P, PD>(v, mmax, fm, tid, nt);
    __syncthreads();
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
    __syncthreads();
    if (sizeof(P) == 4 && A.vec) {
        const int n4 = (N + 3) >> 2;
        for (int i = tid; i < rows * n4; i += nt) {
            const int r2 = i / n4, c = i - r2 * n4;
            *(reinterpret_cast<float4*>(v.out + (size_t)(j0 + r2) * pitch) + c) =
                *reinterpret_cast<const float4*>(rowbuf + (size_t)r2 * sp + 4 * c);
        }
    } else {
        for (int i = tid; i < rows * N; i += nt) {
            const int r2 = i / N, x = i - r2 * N;
            v.out[(size_t)(j0 + r2) * pitch + x] = rowbuf[(size_t)r2 * sp + x];
        }
    }
}

// ---- y-line tile (G columns x C chunks of threads): the operations of k_ysolve_cols ----------
template <typename P, int PD, int B>
__device__ void y_tile(const PersistArgs<P>& A, const FastArgs<P>& a, int z, int arr, int cg, unsigned char* smem,
                       bool restage, int tid, int nt) {
    constexpr int B2 = 8;
    constexpr int NF = FacW<PD>::F, NU = FacW<PD>::U, NS = FacW<PD>::S;
    const Chunks ch = a.ch;
    const int C = ch.C, base = ch.base, G = a.G, mpad = a.mpad;
    const int mmax = base + 2 * PD;
    const FacSmem<P, PD> fm(reinterpret_cast<P*>(smem), mmax);
    P* buf = fm.end();  // [G*C][mpad]
    const bool thr = tid < G * C;
    const int k = thr ? tid / G : 0, c = thr ? tid - k * G : 0;
    const int s = k * base;
    const int m = (k < C - 1) ? base : ch.last;
    const int t = chunk_type(ch, k);
    const int line_raw = cg * G + c;
    const bool valid = thr && line_raw < a.nlines;
    const int line = line_raw < a.nlines ? line_raw : a.nlines - 1;
    const long long off = (long long)z * A.sbytes;
    const LineView<P> v = line_at(a, arr, off);
    const size_t pitch = (size_t)a.pitch;
    P* g = buf + (size_t)(thr ? tid : 0) * mpad;
    if (restage) stage_factors<P, PD>(v, mmax, fm, tid, nt);
    __syncthreads();
    if (thr) {
        const P* Fk = fm.F + t * mmax * NF;
        P prev[PD];
#pragma unroll
        for (int i = 0; i < PD; ++i) prev[i] = P(0);
        const P* src = v.in + (size_t)s * pitch + line;
        int o = 0;
        for (; o + B <= m; o += B) {
            P r[B];
#pragma unroll
            for (int q = 0; q < B; ++q) r[q] = __ldcg(src + q * pitch);
            src += B * pitch;
            fwd_rows<P, PD, B>(r, Fk + o * NF, prev);
#pragma unroll
            for (int q = 0; q < B; ++q) g[o + q] = r[q];
        }
        for (; o < m; ++o) {
            P r[1] = {__ldcg(src)};
            src += pitch;
            fwd_rows<P, PD, 1>(r, Fk + o * NF, prev);
            g[o] = r[0];
        }
        lu_backward<P, PD>(g, m, fm.U + t * mmax * NU);
    }
    __syncthreads();
    if (!valid) return;  // no barrier follows in this tile
    const P* gn = buf + (size_t)((k + 1 < C ? k + 1 : k) * G + c) * mpad;
    const P* gp = buf + (size_t)((k > 0 ? k - 1 : k) * G + c) * mpad + (base - PD);
    P tn[PD], bp[PD];
    interface_solve<P, PD>(ch, k, mmax, fm.S, fm.E, g, g + (base - PD), gn, gp, tn, bp);
    const P* Sk = fm.S + t * mmax * NS;
    const P* bs = v.base ? v.base + (size_t)s * pitch + line : nullptr;
    P* dst = v.out + (size_t)s * pitch + line;
    const P tmax = a.tmax;
    bool bad = false;
    auto finish = [&](auto nrows, int o) {
        constexpr int R = decltype(nrows)::value;
        P x[R], bv[R];
#pragma unroll
        for (int q = 0; q < R; ++q) {
            x[q] = g[o + q];
            bv[q] = bs ? __ldcg(bs + (size_t)q * pitch) : P(0);
        }
        spike_rows<P, PD, R>(x, Sk + o * NS, tn, bp);
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const P y = x[q] + bv[q];
            dst[(size_t)q * pitch] = y;
            bad |= !(fabs(y) <= tmax);
        }
        if (bs) bs += R * pitch;
        dst += R * pitch;
    };
    int o = 0;
    for (; o + B2 <= m; o += B2) finish(std::integral_constant<int, B2>{}, o);
    for (; o < m; ++o) finish(std::integral_constant<int, 1>{}, o);
    if (bad && v.status != nullptr && arr == 0) atomicOr(v.status, WF_STATUS_UNSTABLE);
}

// ---- substep-2 right-hand side tile (one warp): the operations of k_matvec_stream ------------
template <typename P, int PD, int RS>
__device__ void mv_tile(const PersistArgs<P>& A, int z, int item) {
    constexpr int W = 2 * PD + 1, NR = RS + 2 * PD;
    const int lane = threadIdx.x & 31;
    const long long off = (long long)z * A.sbytes;
    const int Nx = A.Nx, Ny = A.Ny;
    const size_t pitch = (size_t)A.pitch;
    const P* T = shift(A.mT, off);
    const P* F = shift(A.mF, off);
    P* R = shift(A.mR, off);
    const P* A1 = shift(A.mA1, off);
    const P* B1 = shift(A.mB1, off);
    const P* A2 = shift(A.mA2, off);
    const P* B2 = shift(A.mB2, off);
    const P Fscale = A.mFscale, c1 = A.mc1, c2 = A.mc2;
    const int sg = item / A.mv_nstrips, st = item - sg * A.mv_nstrips;
    const int x = st * (32 - 2 * PD) - PD + lane;
    const bool xok = x >= 0 && x < Nx;
    const bool out = lane >= PD && lane < 32 - PD && x < Nx;
    const int j0 = sg * RS;
    const bool yint = j0 >= 2 * PD && j0 + RS + 2 * PD <= Ny;
    P tv[NR], fv[RS];
    if (yint) {
        const P* tp = T + (size_t)(j0 - PD) * pitch + (xok ? x : 0);
        const P* fp = F + (size_t)j0 * pitch + (xok ? x : 0);
#pragma unroll
        for (int i = 0; i < NR; ++i) tv[i] = xok ? __ldcg(tp + (size_t)i * pitch) : P(0);
#pragma unroll
        for (int i = 0; i < RS; ++i) fv[i] = out ? __ldcg(fp + (size_t)i * pitch) : P(0);
    } else {
#pragma unroll
        for (int i = 0; i < NR; ++i) {
            const int r = j0 - PD + i;
            tv[i] = (xok && r >= 0 && r < Ny) ? __ldcg(T + (size_t)r * pitch + x) : P(0);
        }
#pragma unroll
        for (int i = 0; i < RS; ++i) {
            const int r = j0 + i;
            fv[i] = (out && r < Ny) ? __ldcg(F + (size_t)r * pitch + x) : P(0);
        }
    }
    P a1v[W], a2v[W];
#pragma unroll
    for (int d = 0; d < W; ++d) {
        a1v[d] = out ? A1[(size_t)x * W + d] : P(0);
        a2v[d] = (out && A2) ? A2[(size_t)x * W + d] : P(0);
    }
    P w1[NR], w2[NR];
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
    if (!out) return;
    if (yint) {
        P b1i[W], b2i[W];
#pragma unroll
        for (int d = 0; d < W; ++d) {
            b1i[d] = c1 * B1[(size_t)(2 * PD) * W + d];
            b2i[d] = A2 ? c2 * B2[(size_t)(2 * PD) * W + d] : P(0);
        }
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
#pragma unroll
        for (int dl = 0; dl < W; ++dl) {
            const P b1 = c1 * B1[(size_t)j * W + dl];
            const P b2 = A2 ? c2 * B2[(size_t)j * W + dl] : P(0);
            acc = fma(b1, w1[o + dl], fma(b2, w2[o + dl], acc));
        }
        R[(size_t)j * pitch + x] = acc;
    }
}

template <int PD>
struct MvRows {
    static constexpr int value = PD > 2 ? 16 : 8;
};

// ---- the kernel ----------------------------------------------------------------------------

// a slot takes part in this step: active and its step budget not spent
template <typename P>
__device__ __forceinline__ bool slot_live(const PersistArgs<P>& A, int z) {
    return ld_relaxed(A.active + z) != 0 && (!A.budget || ld_relaxed(A.budget + z) != 0);
}

// an item of slot z finished; the slot's last item of the step spends one step of its budget
// (every item of the slot has then started, so all of them saw the same budget)
template <typename P>
__device__ __forceinline__ void slot_done(const PersistArgs<P>& A, int* cnt, int z) {
    const int old = atomicAdd(cnt + A.cl.done, 1);
    if (old == A.ctl[3] - 1 && A.budget) {
        const int b = A.budget[z];
        if (b > 0) A.budget[z] = b - 1;
    }
}

// CTAs per SM: four for FP32 with p <= 2 (64 registers: a few spills), else two (128 registers)
template <typename P, int PD>
struct LinesOcc {
    static constexpr int value = (sizeof(P) == 4 && PD <= 2) ? 4 : 2;
};

template <typename P, int PD>
__global__ void __launch_bounds__(kPT, LinesOcc<P, PD>::value) k_lines_persist(const __grid_constant__ PersistArgs<P> A) {
    constexpr int RS = MvRows<PD>::value;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ int s_item, s_go, s_key;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int n = *A.nitems;
    int next = 0;
    if (tid == 0) {
        next = atomicAdd(A.ctl, 1);
        s_key = -1;
    }
    for (;;) {
        if (tid == 0) {
            s_item = next;
            if (next < n) next = atomicAdd(A.ctl, 1);  // fetched while this item runs
        }
        __syncthreads();
        const int it = s_item;
        if (it >= n) break;
        const int4 d = A.items[it];
        const int ph = d.x & 0xff, m = d.x >> 8, z = d.y;  // m: tiles of this item
        int* cnt = A.cnt + (size_t)z * A.cl.stride;
        int* slot_status = shift(A.status, (long long)z * A.sbytes);
        if (tid == 0) {
            // bit 1: the slot takes part in this step; bit 0: go ahead (the inputs of the item's
            // tiles are ready: Y1 and Y2 wait once here; X2 and MV per tile below)
            const bool live = slot_live(A, z);
            bool ok = live && !ld_relaxed(A.ctl + 1);
            if (ok && ph == PH_Y1) ok = wait_count(A, cnt + A.cl.x1 + d.z, A.nxg, slot_status);
            if (ok && ph == PH_Y2) ok = wait_count(A, cnt + A.cl.x2, A.nxg, slot_status);
            s_go = (live ? 2 : 0) | (ok ? 1 : 0);
        }
        const int key = (z << 4) | (ph << 1) | (ph == PH_MV ? 0 : d.z);  // ph <= 4, arr <= 1: bits 0..3
        bool restage = s_key != key;  // read before thread 0 updates it below
        __syncthreads();
        const int go = s_go;
        if (go & 1) {
            if (ph == PH_MV) {
                // warp tiles d.z + warp + 8k, k < m; each waits for the Y1 column groups that cover
                // its strip's columns and halo
                for (int k = 0; k < m; ++k) {
                    const int w = d.z + warp + 8 * k;
                    if (w >= A.mv_nstrips * A.mv_nsegs) break;
                    const int st = w % A.mv_nstrips;
                    const int xlo = max(0, st * (32 - 2 * PD) - PD), xhi = min(A.Nx - 1, st * (32 - 2 * PD) - PD + 31);
                    int ok = 1;
                    if (lane == 0)
                        for (int gq = xlo / A.y1.G; gq <= xhi / A.y1.G && ok; ++gq)
                            ok = wait_count(A, cnt + A.cl.y1col + gq, 1, slot_status) ? 1 : 0;
                    ok = __shfl_sync(0xffffffffu, ok, 0);
                    __syncwarp();  // orders the other lanes' loads after lane 0's acquire
                    if (!ok) break;
                    mv_tile<P, PD, RS>(A, z, w);
                    __syncwarp();
                    if (lane == 0) arrive(cnt + A.cl.mvseg + w / A.mv_nstrips);
                }
            } else {
                const int arr = d.z;
                const bool xd = ph == PH_X1 || ph == PH_X2;
                const FastArgs<P>& a = ph == PH_X1 ? A.x1 : (ph == PH_X2 ? A.x2 : (ph == PH_Y1 ? A.y1 : A.y2));
                for (int k = 0; k < m; ++k) {
                    const int tile = d.w + k;
                    if (ph == PH_X2) {
                        // the MV segments that cover this tile's rows (every strip)
                        if (tid == 0) {
                            const int j0 = tile * a.G, j1 = min(a.nlines, j0 + a.G) - 1;
                            bool ok = true;
                            for (int sgm = j0 / RS; sgm <= j1 / RS && ok; ++sgm)
                                ok = wait_count(A, cnt + A.cl.mvseg + sgm, A.mv_nstrips, slot_status);
                            s_go = ok ? 3 : 2;
                        }
                        __syncthreads();
                        if (!(s_go & 1)) break;
                    }
                    if (xd) {
                        x_tile<P, PD>(A, a, z, arr, tile * a.G, smem, restage, tid, kPT);
                        __syncthreads();
                        if (tid == 0) arrive(cnt + (ph == PH_X1 ? A.cl.x1 + arr : A.cl.x2));
                    } else {
                        y_tile<P, PD, 16>(A, a, z, arr, tile, smem, restage, tid, kPT);
                        __syncthreads();
                        if (tid == 0 && ph == PH_Y1 && arr == 0) arrive(cnt + A.cl.y1col + tile);
                    }
                    restage = false;  // the next tile of the item uses the same factors
                }
                if (tid == 0) s_key = key;
            }
        }
        if (tid == 0 && (go & 2)) slot_done(A, cnt, z);
        __syncthreads();  // s_item, s_key and the shared memory are reused by the next item
    }
}

// ---- host side -----------------------------------------------------------------------------

int sm_count() {
    int sms = 152, dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

// Line-pass kernel arguments of the persistent tiles (compact factors only).
template <typename P, int PD>
bool fill_line(const LineArgs& la, bool xdir, int G_req, FastArgs<P>& f, size_t* smem) {
    const size_t kSmemBudget = (size_t)(220 * 1024) / LinesOcc<P, PD>::value;  // per CTA
    const Chunks& ch = la.f[0].ch;
    for (int q = 0; q < la.narr; ++q)
        if (!la.f[q].compact || la.f[q].ch.base != ch.base || la.f[q].ch.C != ch.C) return false;
    if (ch.C > 32) return false;
    memset(&f, 0, sizeof(f));
    const int mmax = ch.base + 2 * PD;
    const size_t fbytes = (size_t)fac_elems<PD>(mmax) * sizeof(P);
    f.nlines = la.nlines;
    f.pitch = la.pitch;
    f.ch = ch;
    for (int q = 0; q < 2; ++q) {
        f.in[q] = (const P*)la.in[q];
        f.out[q] = (P*)la.out[q];
        f.base[q] = (const P*)la.base[q];
        f.luc[q] = (const P*)la.f[q].luc;
        f.spkc[q] = (const P*)la.f[q].spkc;
        f.Ec[q] = (const P*)la.f[q].Ec;
        f.fpad[q] = nullptr;  // staged element by element (a CTA restages only on a change of operator)
    }
    f.status = la.status;
    f.tmax = (P)la.tmax;
    f.b = la.b;
    f.mpad = (ch.base > ch.last ? ch.base : ch.last) | 1;
    if (xdir) {
        // as the per-pass x pass: lines per warp by the chunk count, the shared-memory row stride
        // spreading a warp's lines over the banks, up to eight warps' lines per tile
        int lsh = ch.C <= 8 ? 3 : (ch.C <= 16 ? 4 : 5);
        if (la.rpw == 1) lsh = 5;
        else if (la.rpw == 2 && lsh < 4) lsh = 4;
        const int lpw = 1 << (5 - lsh);
        const int L = 32 >> (5 - lsh);
        const int slots = sizeof(P) == 4 ? 32 : 16;
        int sp = la.pitch;
        if (L < slots)
            while (sp % (2 * L) != L || (sp * sizeof(P)) % 16 != 0) ++sp;
        int G = (kPT / 32) * lpw;
        if (G_req > 0 && G_req < G) G = (G_req + lpw - 1) / lpw * lpw;
        auto need = [&](int g) { return (size_t)g * sp * sizeof(P) + fbytes; };
        while (G > lpw && need(G) > kSmemBudget) G = ((G / 2) + lpw - 1) / lpw * lpw;
        if (need(G) > kSmemBudget) return false;
        f.G = G;
        f.lsh = lsh;
        f.sp = sp;
        *smem = need(G);
    } else {
        int G = G_req > 0 ? G_req : kPT;
        while (G > 1 && G * ch.C > kPT) G /= 2;
        if (G * ch.C > kPT) return false;
        auto need = [&](int g) { return fbytes + (size_t)g * ch.C * f.mpad * sizeof(P); };
        while (G > 1 && need(G) > kSmemBudget) G /= 2;
        if (need(G) > kSmemBudget) return false;
        f.G = G;
        *smem = need(G);
    }
    return true;
}

template <typename P, int PD>
cudaError_t persist_typed(const PersistHost& h, PersistPlan* plan, bool launch, cudaStream_t s) {
    PersistArgs<P> A;
    memset(&A, 0, sizeof(A));
    size_t sx1 = 0, sy1 = 0, sx2 = 0, sy2 = 0;
    if (!fill_line<P, PD>(h.x1, true, h.xG, A.x1, &sx1) || !fill_line<P, PD>(h.y1, false, h.yG, A.y1, &sy1) ||
        !fill_line<P, PD>(h.x2, true, h.xG, A.x2, &sx2) || !fill_line<P, PD>(h.y2, false, h.yG, A.y2, &sy2))
        return cudaErrorNotSupported;
    if (A.y1.G != A.y2.G || A.x1.G != A.x2.G) return cudaErrorNotSupported;
    constexpr int RS = MvRows<PD>::value;
    A.mT = (const P*)h.mv.T;
    A.mF = (const P*)h.mv.F;
    A.mR = (P*)h.mv.R;
    A.mA1 = (const P*)h.mv.A1;
    A.mB1 = (const P*)h.mv.B1;
    A.mA2 = (const P*)h.mv.A2;
    A.mB2 = (const P*)h.mv.B2;
    A.mFscale = (P)h.mv.Fscale;
    A.mc1 = (P)h.mv.c1;
    A.mc2 = (P)h.mv.c2;
    A.mv_nstrips = (h.mv.Nx + (32 - 2 * PD) - 1) / (32 - 2 * PD);
    A.mv_nsegs = (h.mv.Ny + RS - 1) / RS;
    A.sbytes = h.mv.b.sbytes;
    A.Nx = h.mv.Nx;
    A.Ny = h.mv.Ny;
    A.pitch = h.mv.pitch;
    A.nxg = (h.x1.nlines + A.x1.G - 1) / A.x1.G;
    A.nyg = (h.y1.nlines + A.y1.G - 1) / A.y1.G;
    bool vec = sizeof(P) == 4 && (h.mv.pitch % 4) == 0 && (A.sbytes % 16) == 0;
    for (const LineArgs* la : {&h.x1, &h.x2})
        for (int q = 0; q < la->narr; ++q) vec = vec && ((uintptr_t)la->in[q] % 16 == 0) && ((uintptr_t)la->out[q] % 16 == 0);
    A.vec = vec ? 1 : 0;
    CntLayout cl;
    cl.x1 = 0;
    cl.y1col = cl.x1 + 2;
    cl.mvseg = cl.y1col + A.nyg;
    cl.x2 = cl.mvseg + A.mv_nsegs;
    cl.done = cl.x2 + 1;
    cl.stride = (cl.done + 1 + 31) & ~31;  // 128-byte blocks per slot
    A.cl = cl;
    const size_t smem = std::max(std::max(sx1, sx2), std::max(sy1, sy2));
    auto kern = k_lines_persist<P, PD>;
    cudaError_t e = allow_dynamic_smem(kern, (size_t)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kPT, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorNotSupported;
    plan->nq = 0;
    plan->nmv = A.mv_nstrips * A.mv_nsegs;  // warp tiles
    plan->nxg = A.nxg;
    plan->nyg = A.nyg;
    plan->narr1 = h.x1.narr;
    plan->cstride = cl.stride;
    plan->ctas = per_sm * sm_count();
    plan->seg = 0;
    plan->xG = A.x1.G;
    plan->yG = A.y1.G;
    plan->smem = smem;
    if (!launch) return cudaSuccess;
    // the item list and counters were laid out for this plan (prepare step): never write past them
    if (!h.items || !h.ctl || !h.cnt || (size_t)h.nslots_cap * cl.stride > h.cnt_cap) return cudaErrorInvalidValue;
    A.items = h.items;
    A.nitems = h.ctl + 2;
    A.ctl = h.ctl;
    A.cnt = h.cnt;
    A.wait_ns = h.wait_ns;
    A.status = h.status;
    A.active = h.active;
    A.budget = h.budget;
    // every counter of this step starts at zero (ticket, abort flag, arrival counters)
    e = cudaMemsetAsync(h.ctl, 0, 2 * sizeof(int), s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(h.cnt, 0, (size_t)h.nslots_cap * cl.stride * sizeof(int), s);
    if (e != cudaSuccess) return e;
    const int grid = per_sm * sm_count();
    kern<<<grid, kPT, smem, s>>>(A);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace

bool persist_supported(int prec, int p, int wind_rank) {
    (void)prec;
    (void)wind_rank;
    return p >= 1 && p <= 3;
}

cudaError_t persist_step(const PersistHost& h, PersistPlan* plan, bool launch, cudaStream_t s) {
    PersistPlan dummy;
    if (!plan) plan = &dummy;
#define WF_PS(P, PD) return persist_typed<P, PD>(h, plan, launch, s)
    if (h.prec == 0) {
        switch (h.p) {
            case 1: WF_PS(float, 1);
            case 2: WF_PS(float, 2);
            case 3: WF_PS(float, 3);
        }
    } else {
        switch (h.p) {
            case 1: WF_PS(double, 1);
            case 2: WF_PS(double, 2);
            case 3: WF_PS(double, 3);
        }
    }
#undef WF_PS
    return cudaErrorNotSupported;
}

// Wavefront order of the work items over groups of `gs` active slots (see the top of the file).
// An item covers several consecutive tiles of one (pass, slot, array): about two items per CTA
// in every pass over all active slots, so that a CTA stages an operator's factors once for
// several tiles and the fixed costs of an item (claim, barriers, dependency check) amortise.
int persist_items(const PersistPlan& plan, const int* slots, int nslots, int gs, int4* out, int cap,
                  int* items_per_slot) {
    if (gs < 1) gs = 1;
    const int ngroups = (nslots + gs - 1) / gs;
    const long target = 2L * std::max(1, plan.ctas);
    auto per_item = [&](long tiles_all, int most) {
        return (int)std::max(1L, std::min((long)most, tiles_all / target));
    };
    const int tx = per_item((long)nslots * plan.narr1 * plan.nxg, plan.nxg);
    const int ty = per_item((long)nslots * plan.narr1 * plan.nyg, plan.nyg);
    const int mv8 = (plan.nmv + 7) / 8;  // CTA rounds of eight warp tiles
    const int tm = per_item((long)nslots * mv8, mv8);
    int n = 0, per_slot = 0;
    auto put = [&](int ph, int m, int z, int a, int b) {
        if (n < cap) out[n] = make_int4(ph | (m << 8), z, a, b);
        ++n;
    };
    auto tiles = [&](int ph, int z, int arr, int count, int per) {
        for (int i = 0; i < count; i += per) put(ph, std::min(per, count - i), z, arr, i);
    };
    for (int t = 0; t < ngroups + PH_N - 1; ++t)
        for (int ph = 0; ph < PH_N; ++ph) {
            const int g = t - ph;
            if (g < 0 || g >= ngroups) continue;
            for (int k = g * gs; k < std::min(nslots, (g + 1) * gs); ++k) {
                const int z = slots[k];
                const int n0 = n;
                switch (ph) {
                    case PH_X1:
                        for (int arr = 0; arr < plan.narr1; ++arr) tiles(PH_X1, z, arr, plan.nxg, tx);
                        break;
                    case PH_Y1:
                        for (int arr = 0; arr < plan.narr1; ++arr) tiles(PH_Y1, z, arr, plan.nyg, ty);
                        break;
                    case PH_MV:
                        for (int i = 0; i < mv8; i += tm) put(PH_MV, std::min(tm, mv8 - i), z, 8 * i, 0);
                        break;
                    case PH_X2:
                        tiles(PH_X2, z, 0, plan.nxg, tx);
                        break;
                    case PH_Y2:
                        tiles(PH_Y2, z, 0, plan.nyg, ty);
                        break;
                }
                if (k == 0) per_slot += n - n0;
            }
        }
    *items_per_slot = per_slot;
    return n;
}

}  // namespace wf
