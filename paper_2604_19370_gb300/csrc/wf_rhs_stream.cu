// Explicit right-hand side by sum-factorised Gauss quadrature, streaming form.
//
// Computes exactly what k_rhs (wf_rhs.cu) computes (Eq. termsPR's F tested against
// every basis function, the fuel increment of the Sec. 7 listing and the
// increment-form right-hand side R = Rscale F + c1 (A1 (x) B1) T + c2 (A2 (x) B2) T),
// with a different schedule:
//
//   * one warp owns a strip of 32 element columns (lane L <-> element column
//     X0 - p + L) and walks down a segment of element rows;
//   * everything the sum factorisation needs lives in registers as sliding
//     windows over rows: the x-interpolated values (T, dT/dx, phi) of the p+1
//     coefficient rows an element row uses, the y-test accumulators of the p+1
//     DOF rows it contributes to, and the x-convolved coefficient rows of the
//     explicit Kronecker products;
//   * neighbouring element columns are reached with warp shuffles, so nothing
//     goes through shared memory;
//   * a DOF row is finished (x-test contraction, matvec, stores) as soon as the
//     last element row touching it has been processed;
//   * with uniform knots every element p <= e < n - p has the same B, B' tables; the
//     rows are cut into a segment of the first 2p DOF rows, interior segments and a
//     segment of the last 2p, so that a warp on an interior strip and segment touches
//     interior elements only and takes every table from the kernel's parameter block
//     (constant operands of the FMAs, no registers); in FP32 a warp on a boundary strip
//     of an interior segment holds its element's x tables in registers, and the warps of
//     the boundary segments read their element's tables through L1;
//   * warps take (strip, segment) work items in a flat order, so none idles when the
//     strips of a row do not fill a CTA.
//
// Lanes 0..p-1 only feed their neighbours, so a strip produces 32 - p DOF
// columns; a segment recomputes p element rows above it.  Both overheads are
// below 7 % for p = 2.
#include "wf_rhs_stream.cuh"

namespace wf {

namespace {

// Work items = (strip, segment) of one scenario.  MODE 2: every item, interior segments first and
// the short boundary segments last, each warp taking the fast or the general form.  With
// FP32 the items are split between launches whose register budgets differ: MODE 0 runs the
// interior items (interior strip x interior segment: the packed form with constant tables,
// which needs few registers, so sixteen one-warp CTAs fit an SM), MODE 1 the boundary strips
// of the interior segments in the packed form with x tables in registers (on segments of
// their own, shorter height; sixteen per SM) and MODE 4 the boundary segments in the general
// form (twelve per SM).  One warp per CTA, so that a warp slot frees as soon as its own item
// ends.
// MODE 3 (FP32): the items of MODE 0 followed by those of MODE 1 and MODE 4 in one launch at sixteen
// warps per SM, for a step that must take one launch for its quadrature.
template <typename P, int PD, int WR, int MODE>
struct RhsOcc {
    static constexpr int value = sizeof(P) != 4 || PD > 2 ? 1 : (MODE == 0 || MODE == 3 || MODE == 1 ? 16 : 12);
};

template <typename P, int PD, int WR, int MODE>
__global__ void __launch_bounds__(32, RhsOcc<P, PD, WR, MODE>::value) k_rhs_stream(const StreamArgs<P> a_in) {
    extern __shared__ float wind_rows[];  // FP32 packed form: the item's wind factors
    if (!scene_active(a_in.b)) return;
    StreamArgs<P> a = a_in;
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
    const int lane = threadIdx.x & 31;
    const int item = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int nsi = a.s_hi - a.s_lo;          // interior strips
    const int nseg_in = a.split ? a.nsegs - 2 : 0;  // interior segments (listed first)
    // item -> strip and segment; segments: 0 .. nseg_in-1 interior (height seg), nseg_in the
    // first 2p DOF rows, nseg_in+1 the last 2p (split), or plain pieces of height seg
    int sg, strip, seg = a.seg;
    // MODE 3: the first nsi * nseg_in items as MODE 0, the rest as MODE 1
    const bool as0 = MODE == 0 || (MODE == 3 && item < nsi * nseg_in);
    const int item1 = MODE == 3 ? item - nsi * nseg_in : item;
    if (as0) {
        if (item >= nsi * nseg_in) return;  // whole warp leaves; no block barrier in this kernel
        sg = item / nsi;
        strip = a.s_lo + (item - sg * nsi);
    } else if (MODE == 1 || MODE == 3 || MODE == 4) {
        const int nb = a.nstrips - nsi;      // boundary strips: [0, s_lo) and [s_hi, nstrips)
        const int first = nb * a.nseg_b;     // boundary strips x interior segments of height
        // MODE 1: the boundary strips' items only; MODE 4: the boundary segments' only
        if (MODE == 1 && item1 >= first) return;
        const int item = MODE == 4 ? item1 + first : item1;
        if (item < first) {                  // seg_b, then every strip x the two boundary segments
            sg = item / nb;
            const int bs = item - sg * nb;
            strip = bs < a.s_lo ? bs : a.s_hi + (bs - a.s_lo);
            seg = a.seg_b;
        } else {
            const int g = item - first;
            if (g >= 2 * a.nstrips) return;
            sg = -1 - g / a.nstrips;         // -1: first 2p rows, -2: last 2p rows
            strip = g - (g / a.nstrips) * a.nstrips;
        }
    } else {
        if (item >= a.nstrips * a.nsegs) return;
        sg = item / a.nstrips;
        strip = item - sg * a.nstrips;
        if (a.split && sg >= nseg_in) sg = nseg_in - 1 - sg;  // nseg_in -> -1, nseg_in+1 -> -2
    }
    const int X0 = strip * (32 - PD);
    int Y0, Y1;
    bool yint = false;
    if (!a.split) {
        Y0 = sg * a.seg;
        Y1 = min(Y0 + a.seg, a.Ny);
    } else if (sg >= 0) {
        // interior segments (the long items), element rows Y0 - p .. Y1 - 1 in [p, ny - p)
        Y0 = 2 * PD + sg * seg;
        Y1 = min(Y0 + seg, a.Ny - 2 * PD);
        yint = true;
    } else if (sg == -1) {
        Y0 = 0;
        Y1 = 2 * PD;
    } else {
        Y0 = a.Ny - 2 * PD;
        Y1 = a.Ny;
    }
    const bool xint = a_in.it.xok && X0 >= 2 * PD && X0 + 31 < a.nx;
    if constexpr (sizeof(P) == 4) {
        // FP32: interior strips of interior segments with constant tables (MODE 0), the other
        // strips of interior segments with x tables in registers, boundary segments general.
        // MODE 2 runs in FP32 only where no strip is interior.
        if constexpr (MODE == 1) {
            stream_strip_pairs<PD, WR, true>(a, a_in.it, a_in.pr, lane, X0, Y0, Y1, wind_rows);
        } else if constexpr (MODE == 4) {
            stream_strip<P, PD, WR, false>(a, a_in.it, lane, X0, Y0, Y1);
        } else {
            if (as0)
                stream_strip_pairs<PD, WR, false>(a, a_in.it, a_in.pr, lane, X0, Y0, Y1, wind_rows);
            else if (yint)
                stream_strip_pairs<PD, WR, true>(a, a_in.it, a_in.pr, lane, X0, Y0, Y1, wind_rows);
            else
                stream_strip<P, PD, WR, false>(a, a_in.it, lane, X0, Y0, Y1);
        }
    } else {
        if (xint && yint)
            stream_strip<P, PD, WR, true>(a, a_in.it, lane, X0, Y0, Y1);
        else
            stream_strip<P, PD, WR, false>(a, a_in.it, lane, X0, Y0, Y1);
    }
}


// Dynamic shared memory of a launch whose packed-form items span at most seg + p element rows:
// 2 WR (p+1) wind factors per row (none in FP64 or without wind variation); above the default
// 48 KB the kernel is opted in to more; SIZE_MAX if it cannot be had.
template <typename P, int PD, int WR, int MODE>
size_t wind_smem(int seg) {
    if (sizeof(P) != 4 || WR == 0) return 0;
    const size_t bytes = (size_t)2 * WR * (PD + 1) * (seg + PD) * sizeof(float);
    if (bytes > 48 * 1024) {
        if (bytes > 227 * 1024) return SIZE_MAX;
        if (allow_dynamic_smem(k_rhs_stream<P, PD, WR, MODE>, bytes) != cudaSuccess)
            return SIZE_MAX;
    }
    return bytes;
}

template <typename P, int PD, int WR>
cudaError_t run_stream(const RhsArgs& r, cudaStream_t s) {
    constexpr int WARPS = 1;
    StreamArgs<P> a;
    int sms = 152;
    {
        int dev = 0;
        if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    }
    // segment height: the largest power of two from 128 down to 16 that still gives every
    // resident warp (twelve per SM) an item
    const int nstrips = (r.Nx + (32 - PD) - 1) / (32 - PD);
    int seg = 128;
    while (seg > 16 && (long)nstrips * ((r.Ny + seg - 1) / seg) * r.b.S < 12L * sms) seg /= 2;
    if (r.seg > 0) seg = r.seg;
    fill_stream_args<P, PD>(r, seg, a);
    const int mid = r.Ny - 4 * PD;
    const long n_fast = (long)(a.s_hi - a.s_lo) * (a.split ? a.nsegs - 2 : 0);
    const long n_all = (long)a.nstrips * a.nsegs;
    // the boundary strips' interior segments run beside the interior launch, few of them: they
    // take shorter segments (down to 8 rows) so that four items per SM exist
    {
        const int nb = a.nstrips - (a.s_hi - a.s_lo);
        int sb = seg;
        while (sb / 2 >= 8 && (long)nb * ((mid + sb - 1) / sb) * r.b.S < 4L * sms) sb /= 2;
        a.seg_b = sb;
        a.nseg_b = a.split ? (mid + sb - 1) / sb : 0;
    }
    const long n_side = (long)(a.nstrips - (a.s_hi - a.s_lo)) * a.nseg_b + 2L * a.nstrips;
    // FP32 only (FP64 runs every item in one launch): split launches when interior items exist
    if constexpr (sizeof(P) == 4) {
        if (n_fast > 0 && r.single) {
            // one launch: the interior items, then the others (a step form with one launch for
            // its quadrature)
            const size_t wb3 = wind_smem<P, PD, WR, 3>(a.seg);
            if (wb3 == SIZE_MAX) return cudaErrorInvalidValue;
            dim3 g3((unsigned)((n_fast + n_side + WARPS - 1) / WARPS), 1, r.b.S);
            k_rhs_stream<P, PD, WR, 3><<<g3, 32 * WARPS, wb3, s>>>(a);
            count_launches(1);
            return cudaGetLastError();
        }
        if (n_fast > 0) {
            // interior items in one launch, the rest in a second (their register budgets differ);
            // with the handle's second stream the two run side by side and join before returning
            cudaError_t e;
            const bool fork = r.aux && r.ev_fork && r.ev_join;
            cudaStream_t s1 = fork ? r.aux : s;
            if (fork) {
                if ((e = cudaEventRecord(r.ev_fork, s)) != cudaSuccess) return e;
                if ((e = cudaStreamWaitEvent(r.aux, r.ev_fork, 0)) != cudaSuccess) return e;
            }
            const size_t wb0 = wind_smem<P, PD, WR, 0>(a.seg), wb1 = wind_smem<P, PD, WR, 1>(a.seg_b);
            if (wb0 == SIZE_MAX || wb1 == SIZE_MAX) return cudaErrorInvalidValue;
            // the boundary strips' items (packed form, sixteen warps per SM) and the boundary
            // segments' items (general form, twelve) in launches of their own
            const long n_bstrip = (long)(a.nstrips - (a.s_hi - a.s_lo)) * a.nseg_b, n_bseg = n_side - n_bstrip;
            if (n_bstrip > 0) {
                dim3 g1((unsigned)((n_bstrip + WARPS - 1) / WARPS), 1, r.b.S);
                k_rhs_stream<P, PD, WR, 1><<<g1, 32 * WARPS, wb1, s1>>>(a);
                if ((e = cudaGetLastError()) != cudaSuccess) return e;
                count_launches(1);
            }
            if (n_bseg > 0) {
                dim3 g4((unsigned)((n_bseg + WARPS - 1) / WARPS), 1, r.b.S);
                k_rhs_stream<P, PD, WR, 4><<<g4, 32 * WARPS, 0, s1>>>(a);
                if ((e = cudaGetLastError()) != cudaSuccess) return e;
                count_launches(1);
            }
            dim3 g0((unsigned)((n_fast + WARPS - 1) / WARPS), 1, r.b.S);
            k_rhs_stream<P, PD, WR, 0><<<g0, 32 * WARPS, wb0, s>>>(a);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            count_launches(1);
            if (fork) {
                if ((e = cudaEventRecord(r.ev_join, r.aux)) != cudaSuccess) return e;
                if ((e = cudaStreamWaitEvent(s, r.ev_join, 0)) != cudaSuccess) return e;
            }
            return cudaSuccess;
        }
    }
    dim3 grid((unsigned)((n_all + WARPS - 1) / WARPS), 1, r.b.S);
    const size_t wb2 = wind_smem<P, PD, WR, 2>(a.seg);
    if (wb2 == SIZE_MAX) return cudaErrorInvalidValue;
    k_rhs_stream<P, PD, WR, 2><<<grid, 32 * WARPS, wb2, s>>>(a);
    count_launches(1);
    return cudaGetLastError();
}

template <typename P, int PD>
cudaError_t by_rank(const RhsArgs& r, cudaStream_t s) {
    if constexpr (sizeof(P) == 8 && PD == 3) {
        return cudaErrorNotSupported;  // its register windows spill: tile form
    } else {
        switch (r.wind_rank) {
            case 0: return run_stream<P, PD, 0>(r, s);
            case 1: return run_stream<P, PD, 1>(r, s);
            case 2: return run_stream<P, PD, 2>(r, s);
        }
        return cudaErrorNotSupported;
    }
}

}  // namespace

cudaError_t launch_rhs_stream(int prec, int p, const RhsArgs& r, cudaStream_t s) {
    if (prec == 0) {
        switch (p) {
            case 1: return by_rank<float, 1>(r, s);
            case 2: return by_rank<float, 2>(r, s);
            case 3: return by_rank<float, 3>(r, s);
        }
    } else {
        switch (p) {
            case 1: return by_rank<double, 1>(r, s);
            case 2: return by_rank<double, 2>(r, s);
            case 3: return by_rank<double, 3>(r, s);
        }
    }
    return cudaErrorNotSupported;
}

}  // namespace wf
