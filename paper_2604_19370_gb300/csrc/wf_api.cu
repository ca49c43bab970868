// C ABI of libwf: handle life cycle, state transfer and the time-step driver.
//
// The step sequences follow the schemes of the paper:
//   Peaceman-Rachford, Sec. 3.1 Eq. matrixPR (one explicit F per step, or per substep);
//   Strang + Crank-Nicolson, Sec. 3.2 Eq. matrixCN;
//   explicit L2 projection (the explicit dynamics of Sec. 6), every term at T^n;
//   fuel: explicit Euler L2 projection of the Sec. 7 listing, (M^x (x) M^y) phi^{n+1} = Phi.
// Each 2-D solve (A^x (x) B^y) X = R runs as an x pass (lines of A^x) and a y pass
// (lines of B^y), Sec. 4.  The launches of one step are captured once into a CUDA
// graph and replayed by wf_step.
//
// A handle holds S scenario slots of one grid (S = 1 for wf_create).  Every slot owns
// one block of device memory with the same layout (fields, wind-dependent operator
// bands and factors, wind tables, guard flag); kernels address slot z at
// z * sbytes past slot 0 and skip slots whose active flag is 0, so slots can join and
// leave between steps without re-capturing the graph.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <new>
#include <vector>

#include "wf.h"
#include "wf_internal.h"

using namespace wf;

namespace {

constexpr double kTmax = 1e5;  // guard on |T| (K)
constexpr int kTune = 8;       // tuned launch shapes (wf_autotune)

struct Arena {
    char* base = nullptr;
    size_t off = 0;
    template <typename T>
    T* take(size_t count) {
        off = (off + 255) & ~(size_t)255;
        T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
        off += count * sizeof(T);
        return p;
    }
};

// One directional operator of slot 0 (every other slot: same offsets in its block).
struct Op {
    bool factored = false;
    bool compact = false;
    int mmax = 0;
    double *band64 = nullptr, *lu64 = nullptr, *spk64 = nullptr, *E64 = nullptr;
    void *bandP = nullptr, *luP = nullptr, *spkP = nullptr, *EP = nullptr;
    double *luc64 = nullptr, *spkc64 = nullptr, *Ec64 = nullptr;
    void *lucP = nullptr, *spkcP = nullptr, *EcP = nullptr;
    void* fpadP = nullptr;  // compact factors in the line kernels' padded layout (working precision)
};

struct Dir {
    int n = 0, N = 0;
    double L = 0, h = 0;
    Chunks ch{};
    ElemTabs itab{};  // host copy of the interior element's tables
    // shared by all slots
    double *B64 = nullptr, *D64 = nullptr;
    void *BP = nullptr, *DP = nullptr, *wP = nullptr;
    double *M64 = nullptr, *K64 = nullptr, *G64 = nullptr;
    // per slot
    Op op[3];  // 0: M, 1: -theta A (explicit side, band only), 2: M + theta A (implicit side)
};

// Host-side settings of one slot.
struct Slot {
    double wind_x = 0, wind_y = 0;
    int wind_rank = 0;
    bool active = false;
    double coef[2][3][3] = {};  // [dir][op][aM, aK, aG]
};

enum SiteId { S_RHS1, S_X1, S_Y1, S_Y2PRE, S_RHS2, S_MV2, S_X2, S_Y3, S_PERSIST, S_NSITES };
const char* kSiteNames[S_NSITES] = {"rhs_quadrature_1", "xsolve_1", "ysolve_1", "ysolve_y_substep",
                                    "rhs_quadrature_2", "matvec_2", "xsolve_2", "ysolve_2",
                                    "step_persistent"};

}  // namespace

struct wf_handle {
    int nx, ny, p, q, Nx, Ny, pitch, prec;
    double dt;
    wf_params prm;
    Phys phys;
    cudaStream_t own = nullptr, stream = nullptr;
    // second stream: the quadrature's boundary items run there beside its interior items
    cudaStream_t aux = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // step form 3: the slots in two groups, the second group's launches on stream gs; while a
    // launch runs over one group (gn > 0) its kernels see slots gz0 .. gz0+gn-1 (the per-slot
    // pointers then point at slot gz0's block), and ev_rhs (if set) is recorded after the group's
    // first quadrature
    cudaStream_t gs = nullptr;
    cudaEvent_t ev_q = nullptr, ev_g = nullptr, ev_rhs = nullptr;
    int gz0 = 0, gn = 0;
    // wf_batch_run: upload and download streams, and events (per group: uploaded, done; a start
    // and an end event), created on the first call
    cudaStream_t io_in = nullptr, io_out = nullptr;
    cudaEvent_t ev_io[18] = {};
    void* mem = nullptr;
    size_t mem_bytes = 0;
    // shared region
    double *gxi = nullptr, *gw = nullptr;
    double* stage = nullptr;   // 2 * Nx * Ny doubles for host transfers
    void* bstage = nullptr;    // whole-batch host transfers (allocated on first use)
    size_t bstage_bytes = 0;
    double* work64 = nullptr;
    double* diag = nullptr;    // [4] factorisation diagnostics
    double* wind64 = nullptr;  // staging of wind factors
    int* active_dev = nullptr;
    int* budget_dev = nullptr;  // [S] step budgets (wf_batch_set_budget; -1: unlimited)
    bool budget_on = false;     // some budget was set: the step spends them
    int* status_out = nullptr;  // [S] gathered guard flags
    Dir dx, dy;
    // slot blocks: slot-0 pointers, block stride
    int S = 1;
    long long sbytes = 0;
    char* slots_mem = nullptr;  // start of slot 0's block
    long long wait_ns = 1000000000LL;  // limit of every bounded device wait (wf_set_wait_limit)
    bool mms_on = false;       // manufactured-solution forcing (wf_set_mms)
    MmsArgs mms{};
    double* tdev = nullptr;    // device: start time of the next step (advanced only with forcing)
    int tune[kTune] = {0, 0, 0, 0, 0, 0, 0, 0};  // x lines per CTA (first x pass), y lines per CTA,
                                           // quadrature segment rows, x lines per warp, x lines
                                           // per CTA of the second x pass, its right-hand side
                                           // (1 fused, 2 separate matvec), step form (1 per-pass
                                           // launches, 2 persistent), slots per group of the
                                           // persistent order (0: the launchers' rules)
    // persistent step: work items, ticket / abort / item count, arrival counters (allocated on
    // first use); the item list is rebuilt when the active slots or the shapes change
    int4* p_items = nullptr;
    int* p_ctl = nullptr;
    int* p_cnt = nullptr;
    size_t p_items_cap = 0, p_cnt_cap = 0;
    bool p_dirty = true;
    bool noalloc_run = false;  // wf_step_noalloc in progress: per-pass launches only
    void *T = nullptr, *phi = nullptr, *F = nullptr, *Phi = nullptr, *R = nullptr;
    int* status = nullptr;
    void *fxq = nullptr, *gxq = nullptr, *fyq = nullptr, *gyq = nullptr;
    std::vector<Slot> slots;
    std::vector<int> active_host;
    bool active_dirty = true;
    int wr = 0;  // wind rank the kernels are launched with (max over slots)
    cudaGraphExec_t g1 = nullptr, g8 = nullptr;
    bool profiling = false;
    std::vector<cudaEvent_t> ev_free;
    struct Pending {
        int site;
        cudaEvent_t a, b;
    };
    std::vector<Pending> pending;
    double site_ms[S_NSITES] = {0};
    int site_cnt[S_NSITES] = {0};
};

namespace wf {
std::atomic<unsigned long long> g_launches{0};
void count_launches(int n) { g_launches.fetch_add((unsigned long long)n, std::memory_order_relaxed); }
}  // namespace wf

namespace {

#define WF_TRY(expr)                            \
    do {                                        \
        cudaError_t _e = (expr);                \
        if (_e != cudaSuccess) return WF_ECUDA; \
    } while (0)

size_t esize(int prec) { return prec == WF_FP32 ? 4 : 8; }

template <typename T>
T* at(const wf_handle* h, T* p, int slot) {
    return p ? reinterpret_cast<T*>(reinterpret_cast<char*>(const_cast<void*>(static_cast<const void*>(p))) +
                                    (long long)slot * h->sbytes)
             : p;
}

Batch batch(const wf_handle* h) {
    // a launch over a slot group: the group's flags (its per-slot pointers are rebased by
    // rebase_slots)
    const int z0 = h->gn > 0 ? h->gz0 : 0;
    Batch b;
    b.S = h->gn > 0 ? h->gn : h->S;
    b.sbytes = h->sbytes;
    b.active = h->active_dev + z0;
    b.budget = h->budget_on ? h->budget_dev + z0 : nullptr;
    return b;
}

// Chunks of length `base`; the last chunk takes the remainder and is merged into its
// neighbour when it would be shorter than 2p, so every chunk holds at least 2p rows
// and the interior chunks (1 .. C-2) lie entirely in the Toeplitz part of the operator.
Chunks make_chunks(int N, int base, int p) {
    Chunks c;
    c.N = N;
    c.base = base;
    c.C = (N + base - 1) / base;
    c.last = N - (c.C - 1) * base;
    if (c.C > 1 && c.last < 2 * p) {
        c.C -= 1;
        c.last += base;
    }
    if (c.C == 1) c.last = N;
    return c;
}

void layout_shared(wf_handle* h, Arena& A) {
    h->stage = A.take<double>(2 * (size_t)h->Nx * h->Ny);
    h->gxi = A.take<double>(16);
    h->gw = A.take<double>(16);
    h->diag = A.take<double>(4);
    h->active_dev = A.take<int>(h->S);
    h->budget_dev = A.take<int>(h->S);
    h->status_out = A.take<int>(h->S);
    h->tdev = A.take<double>(1);
    const int W = 2 * h->p + 1;
    const int maxN = h->Nx > h->Ny ? h->Nx : h->Ny;
    h->work64 = A.take<double>((size_t)maxN * W);
    h->wind64 = A.take<double>((size_t)2 * kMaxRank * (h->Nx + h->Ny));
    Dir* ds[2] = {&h->dx, &h->dy};
    for (Dir* d : ds) {
        const size_t tab = (size_t)d->n * h->q * (h->p + 1);
        d->B64 = A.take<double>(tab);
        d->D64 = A.take<double>(tab);
        if (h->prec == WF_FP32) {
            d->BP = A.take<float>(tab);
            d->DP = A.take<float>(tab);
            d->wP = A.take<float>(16);
        } else {
            d->BP = d->B64;
            d->DP = d->D64;
            d->wP = A.take<double>(16);
        }
        d->M64 = A.take<double>((size_t)d->N * W);
        d->K64 = A.take<double>((size_t)d->N * W);
        d->G64 = A.take<double>((size_t)d->N * W);
    }
}

// Slot block, laid out relative to its own start (A.base = start of slot 0).
void layout_slot(wf_handle* h, Arena& A) {
    const size_t es = esize(h->prec);
    const size_t field = (size_t)h->Ny * h->pitch;
    h->T = A.take<char>(field * es);
    h->phi = A.take<char>(field * es);
    h->F = A.take<char>(field * es);
    h->Phi = A.take<char>(field * es);
    h->R = A.take<char>(field * es);
    h->status = A.take<int>(4);
    const int W = 2 * h->p + 1;
    Dir* ds[2] = {&h->dx, &h->dy};
    for (Dir* d : ds) {
        for (Op& o : d->op) {
            const size_t nE = (size_t)(d->ch.C > 1 ? d->ch.C - 1 : 1) * h->p * h->p;
            o.mmax = d->ch.base + 2 * h->p;
            o.band64 = A.take<double>((size_t)d->N * W);
            o.lu64 = A.take<double>((size_t)d->N * W);
            o.spk64 = A.take<double>((size_t)d->N * 2 * h->p);
            o.E64 = A.take<double>(nE);
            o.luc64 = A.take<double>((size_t)3 * o.mmax * W);
            o.spkc64 = A.take<double>((size_t)3 * o.mmax * 2 * h->p);
            o.Ec64 = A.take<double>((size_t)3 * h->p * h->p);
            if (h->prec == WF_FP32) {
                o.bandP = A.take<float>((size_t)d->N * W);
                o.luP = o.factored ? (void*)A.take<float>((size_t)d->N * W) : nullptr;
                o.spkP = o.factored ? (void*)A.take<float>((size_t)d->N * 2 * h->p) : nullptr;
                o.EP = o.factored ? (void*)A.take<float>(nE) : nullptr;
                o.lucP = o.factored ? (void*)A.take<float>((size_t)3 * o.mmax * W) : nullptr;
                o.spkcP = o.factored ? (void*)A.take<float>((size_t)3 * o.mmax * 2 * h->p) : nullptr;
                o.EcP = o.factored ? (void*)A.take<float>((size_t)3 * h->p * h->p) : nullptr;
            } else {
                o.bandP = o.band64;
                o.luP = o.lu64;
                o.spkP = o.spk64;
                o.EP = o.E64;
                o.lucP = o.luc64;
                o.spkcP = o.spkc64;
                o.EcP = o.Ec64;
            }
            o.fpadP = o.factored ? (void*)A.take<char>(fac_pad_elems(h->p, o.mmax) * es) : nullptr;
        }
    }
    const size_t qx = (size_t)kMaxRank * h->nx * h->q, qy = (size_t)kMaxRank * h->ny * h->q;
    h->fxq = A.take<char>(qx * es);
    h->gxq = A.take<char>(qy * es);
    h->fyq = A.take<char>(qx * es);
    h->gyq = A.take<char>(qy * es);
}

// Operator coefficients of a slot for its mean wind:
//   x: A_x = C_d K + c_W b_x G + c_chi M;  op1 = -theta A_x (band),  op2 = X_+ = M + theta A_x
//   y: A_y = C_d K + c_W b_y G;            op1 = -theta A_y (band),  op2 = Y_+ = M + theta A_y
void set_slot_coeffs(const wf_handle* h, Slot& s) {
    const Phys& c = h->phys;
    const double tau = h->dt;
    // explicit: the "-theta A" operators carry the full tau (the "+" side is not used)
    const bool ex = h->prm.scheme == WF_EXPLICIT;
    const double thx = ex ? tau : (h->prm.scheme == WF_PR ? 0.5 * tau : 0.25 * tau);
    const double thy = ex ? tau : 0.5 * tau;
    double(*x)[3] = s.coef[0];
    double(*y)[3] = s.coef[1];
    x[0][0] = 1.0, x[0][1] = 0.0, x[0][2] = 0.0;
    x[1][0] = -thx * c.c_chi, x[1][1] = -thx * c.C_d, x[1][2] = -thx * c.c_W * s.wind_x;
    x[2][0] = 1.0 + thx * c.c_chi, x[2][1] = thx * c.C_d, x[2][2] = thx * c.c_W * s.wind_x;
    y[0][0] = 1.0, y[0][1] = 0.0, y[0][2] = 0.0;
    y[1][0] = 0.0, y[1][1] = -thy * c.C_d, y[1][2] = -thy * c.c_W * s.wind_y;
    y[2][0] = 1.0, y[2][1] = thy * c.C_d, y[2][2] = thy * c.c_W * s.wind_y;
}

Phys make_phys(const wf_params& p) {
    Phys c;
    const double inv = 1.0 / (p.rho * p.cp);
    c.C_d = p.kappa * inv;
    c.C_nld = 4.0 * p.sigma * p.eps * p.delta_x * inv;
    c.c_rad = p.sigma * p.eps / p.delta_z * inv;
    c.c_chi = p.chi * inv;
    c.c_W = p.cW;
    c.K_ign = -p.heat_scale * p.rho * p.ch * p.hc * p.M_ratio * p.A_r * inv;
    c.k_f = p.fuel_rate * p.A_r;
    c.T_a = p.T_a;
    c.T_amb = p.T_amb;
    c.T_ig = p.T_ig;
    c.phi_min = p.fuel_thresh + p.thresh_guard;
    c.heat_by_fuel = p.scale_heat_by_fuel ? 1 : 0;
    return c;
}

bool params_ok(const wf_params& p) {
    const double v[] = {p.Lx, p.Ly, p.rho, p.cp};
    for (double x : v)
        if (!(x > 0.0) || !isfinite(x)) return false;
    const double w[] = {p.kappa, p.sigma, p.eps, p.ch, p.hc, p.cW, p.chi, p.T_amb, p.T_ig, p.delta_x,
                        p.A_r, p.M_ratio, p.T_a, p.heat_scale, p.fuel_rate, p.fuel_thresh, p.thresh_guard,
                        p.wind_x, p.wind_y};
    for (double x : w)
        if (!isfinite(x)) return false;
    if (!(p.delta_z > 0.0)) return false;  // may be +inf (no vertical radiation)
    if (p.scheme != WF_PR && p.scheme != WF_STRANG_CN && p.scheme != WF_EXPLICIT) return false;
    if (p.precision != WF_FP32 && p.precision != WF_FP64) return false;
    if (p.F_timing != WF_F_ONCE && p.F_timing != WF_F_PER_SUBSTEP) return false;
    return true;
}

int build_tables(wf_handle* h) {
    cudaStream_t s = h->stream;
    WF_TRY(launch_gauss(h->gxi, h->gw, h->q, s));
    Dir* ds[2] = {&h->dx, &h->dy};
    for (Dir* d : ds) {
        WF_TRY(launch_basis(h->gxi, h->q, d->n, h->p, d->L, d->B64, d->D64, s));
        WF_TRY(launch_assemble(d->B64, d->D64, h->gw, h->q, d->n, h->p, d->h, d->M64, d->K64, d->G64, s));
        const size_t tab = (size_t)d->n * h->q * (h->p + 1);
        if (h->prec == WF_FP32) {
            WF_TRY(launch_to_f32(d->B64, (float*)d->BP, tab, s));
            WF_TRY(launch_to_f32(d->D64, (float*)d->DP, tab, s));
        }
    }
    double w[16];
    WF_TRY(cudaMemcpyAsync(w, h->gw, sizeof(double) * h->q, cudaMemcpyDeviceToHost, s));
    WF_TRY(cudaStreamSynchronize(s));
    for (Dir* d : ds) {
        if (h->prec == WF_FP32) {
            float wf32[16];
            for (int a = 0; a < h->q; ++a) wf32[a] = (float)(w[a] * d->h);
            WF_TRY(cudaMemcpyAsync(d->wP, wf32, sizeof(float) * h->q, cudaMemcpyHostToDevice, s));
        } else {
            double w64[16];
            for (int a = 0; a < h->q; ++a) w64[a] = w[a] * d->h;
            WF_TRY(cudaMemcpyAsync(d->wP, w64, sizeof(double) * h->q, cudaMemcpyHostToDevice, s));
        }
        WF_TRY(cudaStreamSynchronize(s));  // the host weight arrays go out of scope
        // interior element p (uniform knots): its tables, read back once
        ElemTabs& it = d->itab;
        memset(&it, 0, sizeof(it));
        for (int a = 0; a < h->q; ++a) it.w[a] = w[a] * d->h;
        it.ok = d->n > 2 * h->p;
        if (it.ok) {
            const int Q = h->q, NB = h->p + 1;
            double tb[16], td[16];
            const size_t off = (size_t)h->p * Q * NB;
            WF_TRY(cudaMemcpyAsync(tb, d->B64 + off, sizeof(double) * Q * NB, cudaMemcpyDeviceToHost, s));
            WF_TRY(cudaMemcpyAsync(td, d->D64 + off, sizeof(double) * Q * NB, cudaMemcpyDeviceToHost, s));
            WF_TRY(cudaStreamSynchronize(s));
            for (int a = 0; a < Q; ++a)
                for (int k = 0; k < NB; ++k) {
                    it.B[a][k] = tb[a * NB + k];
                    it.D[a][k] = td[a * NB + k];
                }
        }
        // an interior row of the mass matrix (assembled from the same element tables)
        const int W = 2 * h->p + 1;
        if (d->N >= 4 * h->p + 1) {
            WF_TRY(cudaMemcpyAsync(it.Mb, d->M64 + (size_t)(2 * h->p) * W, sizeof(double) * W,
                                   cudaMemcpyDeviceToHost, s));
            WF_TRY(cudaStreamSynchronize(s));
        }
    }
    return WF_OK;
}

// Bands and chunked factors of every operator of one slot.  Returns WF_OK, WF_ESINGULAR or
// WF_ETRUNC (neglected spike entries above tol); *worst receives the largest of them.
int build_factors(wf_handle* h, int slot, double tol, double* worst) {
    cudaStream_t s = h->stream;
    const int W = 2 * h->p + 1, S2 = 2 * h->p;
    *worst = 0.0;
    Dir* ds[2] = {&h->dx, &h->dy};
    for (int dd = 0; dd < 2; ++dd) {
        Dir* d = ds[dd];
        for (int k = 0; k < 3; ++k) {
            Op& o = d->op[k];
            const double* cf = h->slots[slot].coef[dd][k];
            double zero[4] = {0.0, 0.0, 0.0, 0.0};
            WF_TRY(cudaMemcpyAsync(h->diag, zero, sizeof(zero), cudaMemcpyHostToDevice, s));
            WF_TRY(launch_factor(d->M64, d->K64, d->G64, cf[0], cf[1], cf[2], d->N, h->p, d->ch,
                                 at(h, o.band64, slot), at(h, o.lu64, slot), at(h, o.spk64, slot),
                                 at(h, o.E64, slot), h->work64, h->diag, s));
            WF_TRY(launch_compact(at(h, o.lu64, slot), at(h, o.spk64, slot), at(h, o.E64, slot), h->p, d->ch,
                                  o.mmax, at(h, o.luc64, slot), at(h, o.spkc64, slot), at(h, o.Ec64, slot), h->diag,
                                  s));
            double dg[4];
            WF_TRY(cudaMemcpyAsync(dg, h->diag, sizeof(dg), cudaMemcpyDeviceToHost, s));
            WF_TRY(cudaStreamSynchronize(s));
            if (o.factored) {
                if (dg[0] != 0.0) return WF_ESINGULAR;
                if (dg[1] > *worst) *worst = dg[1];
                // every slot must agree on the form the kernels read; slot 0 decides at create
                if (slot == 0)
                    o.compact = dg[2] == 0.0;
                else if (o.compact && dg[2] != 0.0)
                    return WF_ETRUNC;
            }
            if (h->prec != WF_FP32) continue;
            const size_t nE = (size_t)(d->ch.C > 1 ? d->ch.C - 1 : 1) * h->p * h->p;
            WF_TRY(launch_to_f32(at(h, o.band64, slot), (float*)at(h, o.bandP, slot), (size_t)d->N * W, s));
            if (o.factored) {
                WF_TRY(launch_to_f32(at(h, o.lu64, slot), (float*)at(h, o.luP, slot), (size_t)d->N * W, s));
                WF_TRY(launch_to_f32(at(h, o.spk64, slot), (float*)at(h, o.spkP, slot), (size_t)d->N * S2, s));
                WF_TRY(launch_to_f32(at(h, o.E64, slot), (float*)at(h, o.EP, slot), nE, s));
                WF_TRY(launch_to_f32(at(h, o.luc64, slot), (float*)at(h, o.lucP, slot), (size_t)3 * o.mmax * W, s));
                WF_TRY(launch_to_f32(at(h, o.spkc64, slot), (float*)at(h, o.spkcP, slot), (size_t)3 * o.mmax * S2,
                                     s));
                WF_TRY(launch_to_f32(at(h, o.Ec64, slot), (float*)at(h, o.EcP, slot), (size_t)3 * h->p * h->p, s));
            }
        }
    }
    for (Dir* d : ds)
        for (Op& o : d->op)
            if (o.factored)
                WF_TRY(launch_pad_factors(h->prec, h->p, o.mmax, at(h, o.lucP, slot), at(h, o.spkcP, slot),
                                          at(h, o.EcP, slot), at(h, o.fpadP, slot), s));
    WF_TRY(cudaStreamSynchronize(s));
    return *worst > tol ? WF_ETRUNC : WF_OK;
}

double trunc_tol(const wf_handle* h) { return h->prec == WF_FP32 ? 1e-8 : 1e-15; }

FactorV fv(const Op& o, const Chunks& ch) {
    FactorV f;
    f.ch = ch;
    f.lu = o.luP;
    f.spk = o.spkP;
    f.E = o.EP;
    f.compact = o.compact ? 1 : 0;
    f.mmax = o.mmax;
    f.luc = o.lucP;
    f.spkc = o.spkcP;
    f.Ec = o.EcP;
    f.fpad = o.compact ? o.fpadP : nullptr;
    return f;
}

cudaEvent_t take_event(wf_handle* h) {
    if (!h->ev_free.empty()) {
        cudaEvent_t e = h->ev_free.back();
        h->ev_free.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

template <typename F>
cudaError_t timed(wf_handle* h, int site, F&& launch) {
    if (!h->profiling) return launch();
    cudaEvent_t a = take_event(h), b = take_event(h);
    cudaEventRecord(a, h->stream);
    cudaError_t e = launch();
    cudaEventRecord(b, h->stream);
    if (e == cudaSuccess) h->pending.push_back({site, a, b});
    else {
        // nothing launched (or the launch failed): the events time no kernel
        cudaEventSynchronize(b);
        h->ev_free.push_back(a);
        h->ev_free.push_back(b);
    }
    return e;
}

// R = Rscale F + c1 (A1 (x) B1) T + c2 (A2 (x) B2) T  (A2 == nullptr drops the second term)
RhsArgs rhs_args(wf_handle* h, const void* T, void* F, void* Phi, void* R, double Rscale, const Op& A1,
                 const Op& B1, double c1, const Op* A2, const Op* B2, double c2) {
    RhsArgs a;
    a.nx = h->nx;
    a.ny = h->ny;
    a.Nx = h->Nx;
    a.Ny = h->Ny;
    a.pitch = h->pitch;
    a.T = T;
    a.phi = h->phi;
    a.F = F;
    a.Phi = Phi;
    a.R = R;
    a.Bx = h->dx.BP;
    a.Dx = h->dx.DP;
    a.By = h->dy.BP;
    a.Dy = h->dy.DP;
    a.wx = h->dx.wP;
    a.wy = h->dy.wP;
    a.wind_rank = h->wr;
    a.fxq = h->fxq;
    a.gxq = h->gxq;
    a.fyq = h->fyq;
    a.gyq = h->gyq;
    a.A1 = A1.bandP;
    a.B1 = B1.bandP;
    a.A2 = A2 ? A2->bandP : nullptr;
    a.B2 = B2 ? B2->bandP : nullptr;
    a.Rscale = Rscale;
    a.c1 = c1;
    a.c2 = c2;
    a.tau = h->dt;
    a.seg = h->tune[2];
    // the boundary items' stream (both slot groups of step form 3 fork to it in turn: a group's
    // quadrature joins back before its line passes, and group B's starts after group A's)
    a.aux = h->aux;
    a.ev_fork = h->ev_fork;
    a.ev_join = h->ev_join;
    a.single = 0;
    a.tx = h->dx.itab;
    a.ty = h->dy.itab;
    a.phys = h->phys;
    a.b = batch(h);
    return a;
}

// xsite: 1 or 2 for the first or second x pass of a step, 0 for a y pass
LineArgs line_args(wf_handle* h, int xsite) {
    const bool xdir = xsite != 0;
    LineArgs a;
    memset(&a, 0, sizeof(a));
    a.nlines = xdir ? h->Ny : h->Nx;
    a.G = xsite == 1 ? h->tune[0] : (xsite == 2 ? h->tune[4] : h->tune[1]);
    a.rpw = xdir ? h->tune[3] : 0;
    a.pitch = h->pitch;
    a.tmax = kTmax;
    a.tstatus = h->status;
    a.wait_ns = h->wait_ns;
    // every y pass of a step reads a right-hand side that the step writes again before its next use
    a.in_dead = xdir ? 0 : 1;
    a.b = batch(h);
    return a;
}

void add_line(LineArgs& a, const void* in, void* out, const Op& o, const Chunks& ch, const void* base = nullptr,
              const void* premul = nullptr, double prescale = 1.0) {
    a.in[a.narr] = in;
    a.out[a.narr] = out;
    a.f[a.narr] = fv(o, ch);
    a.base[a.narr] = base;
    a.premul[a.narr] = premul;
    a.prescale[a.narr] = prescale;
    a.narr++;
}

cudaError_t upload_active(wf_handle* h) {
    if (!h->active_dirty) return cudaSuccess;
    h->p_dirty = true;  // the persistent item list holds the active slots
    cudaError_t e = cudaMemcpyAsync(h->active_dev, h->active_host.data(), sizeof(int) * h->S, cudaMemcpyHostToDevice,
                                    h->stream);
    if (e != cudaSuccess) return e;
    e = cudaStreamSynchronize(h->stream);  // the host copy may change right after
    if (e == cudaSuccess) h->active_dirty = false;
    return e;
}

// Enqueue one time step of every active slot on h->stream.
//
// Every substep is solved for its increment: with X_+ = M + theta A_x and
// Y_+ = M + theta A_y, the PR systems of Eq. matrixPR are identical to
//   (X_+ (x) M^y) (T* - T^n)      = theta F - theta (A_x (x) M^y) T^n - theta (M^x (x) A_y) T^n
//   (M^x (x) Y_+) (T^{n+1} - T*)  = theta F - theta (A_x (x) M^y) T*  - theta (M^x (x) A_y) T*
// and the Strang/Crank-Nicolson systems of Eq. matrixCN to
//   (X_+ (x) M^y) (T* - T^n)      = tau/2 F(T^n) - 2 theta_x (A_x (x) M^y) T^n        (theta_x = tau/4)
//   (I (x) Y_+) (T** - T*)        = -2 theta_y (I (x) A_y) T*                         (theta_y = tau/2)
//   (X_+ (x) M^y) (T^{n+1} - T**) = tau/2 F(T**) - 2 theta_x (A_x (x) M^y) T**
// Rounding errors then scale with the increment instead of the temperature,
// which keeps the FP32 path accurate through the inverse mass matrices.
// quadrature launch, then (with a manufactured solution) its forcing: out1 += s1 int f B,
// out2 += s2 int f B
cudaError_t rhs_and_forcing(wf_handle* h, const RhsArgs& r, void* out1, double s1, void* out2, double s2) {
    cudaError_t e = launch_rhs(h->prec, h->p, r, h->stream);
    if (e != cudaSuccess || !h->mms_on) return e;
    return launch_forcing(h->prec, h->mms, out1, s1, out2, s2, h->stream);
}

cudaError_t enqueue_step_body(wf_handle* h);
void drop_graphs(wf_handle* h);

// The persistent form (one quadrature launch, then one launch over every line pass of every active
// slot) takes PR with one F per step; tuning value 6 picks it (2) or the per-pass launches (1,
// and the rule 0: measured faster on the ensemble and on a single domain).
bool use_persist(const wf_handle* h) {
    // (a launch over a group of slots, gn > 0, takes the per-pass form: the persistent plan lists
    // every active slot of the handle)
    if (h->noalloc_run || h->gn > 0 || h->prm.scheme != WF_PR || h->prm.F_timing != WF_F_ONCE) return false;
    if (!persist_supported(h->prec, h->p, h->wr)) return false;
    return h->tune[6] == 2;
}

// Arguments of the persistent step: those of the per-pass launches of the same step.
void persist_args(wf_handle* h, PersistHost* ph) {
    Op* X = h->dx.op;
    Op* Y = h->dy.op;
    const Chunks& cx = h->dx.ch;
    const Chunks& cy = h->dy.ch;
    const double th = 0.5 * h->dt;
    memset(ph, 0, sizeof(*ph));
    ph->prec = h->prec;
    ph->p = h->p;
    ph->x1 = line_args(h, 1);
    add_line(ph->x1, h->R, h->R, X[2], cx);
    add_line(ph->x1, h->Phi, h->Phi, X[0], cx);
    ph->y1 = line_args(h, 0);
    add_line(ph->y1, h->R, h->T, Y[0], cy, h->T);
    add_line(ph->y1, h->Phi, h->phi, Y[0], cy, h->phi);
    MatvecArgs& mv = ph->mv;
    mv.Nx = h->Nx;
    mv.Ny = h->Ny;
    mv.pitch = h->pitch;
    mv.T = h->T;
    mv.F = h->F;
    mv.R = h->R;
    mv.A1 = X[1].bandP;
    mv.B1 = Y[0].bandP;
    mv.A2 = X[0].bandP;
    mv.B2 = Y[1].bandP;
    mv.Fscale = th;
    mv.c1 = 1.0;
    mv.c2 = 1.0;
    mv.b = batch(h);
    ph->x2 = line_args(h, 2);
    add_line(ph->x2, h->R, h->R, X[0], cx);
    ph->y2 = line_args(h, 0);
    add_line(ph->y2, h->R, h->T, Y[2], cy, h->T);
    ph->y2.status = h->status;
    ph->xG = h->tune[0];
    ph->yG = h->tune[1];
    ph->nslots_cap = h->S;
    ph->wait_ns = h->wait_ns;
    ph->status = h->status;
    ph->items = h->p_items;
    ph->cnt_cap = h->p_cnt_cap;
    ph->ctl = h->p_ctl;
    ph->cnt = h->p_cnt;
    ph->active = h->active_dev;
    ph->budget = h->budget_on ? h->budget_dev : nullptr;
}

// Slots per group of the persistent order.  The rule is one group (the passes in order): groups
// small enough for five of them to stay in L2 leave too few items per pass to fill the GPU, and
// their tiles then wait on one another (measured on the 256-slot ensemble).
int persist_group(const wf_handle* h) {
    if (h->tune[7] > 0) return h->tune[7];
    return h->S;
}

// Allocate the persistent buffers and upload the item list of the active slots when needed.
// Must run outside stream capture (it allocates and synchronises).  Returns WF_OK when the
// step uses the per-pass launches.
int prepare_persist(wf_handle* h) {
    if (!use_persist(h) || !h->p_dirty) return WF_OK;
    PersistHost ph;
    persist_args(h, &ph);
    PersistPlan plan;
    cudaError_t e = persist_step(ph, &plan, false, h->stream);
    if (e == cudaErrorNotSupported) {
        cudaGetLastError();
        h->tune[6] = 1;  // this handle's arguments do not fit the persistent form
        return WF_OK;
    }
    if (e != cudaSuccess) return WF_ECUDA;
    std::vector<int> act;
    for (int z = 0; z < h->S; ++z)
        if (h->active_host[z]) act.push_back(z);
    // room for every slot active, so that slots joining later need no reallocation
    // at most one item per tile
    const size_t most = (size_t)plan.narr1 * (plan.nxg + plan.nyg) + (plan.nmv + 7) / 8 + plan.nxg + plan.nyg;
    const size_t cap = std::max<size_t>(1, (size_t)h->S * most);
    const size_t need_cnt = (size_t)h->S * plan.cstride;
    if (cap > h->p_items_cap || need_cnt > h->p_cnt_cap || !h->p_ctl) {
        if (cudaStreamSynchronize(h->stream) != cudaSuccess) return WF_ECUDA;
        if (h->p_items) cudaFree(h->p_items);
        if (h->p_cnt) cudaFree(h->p_cnt);
        if (h->p_ctl) cudaFree(h->p_ctl);
        h->p_items = nullptr;
        h->p_cnt = nullptr;
        h->p_ctl = nullptr;
        h->p_items_cap = h->p_cnt_cap = 0;
        if (cudaMalloc(&h->p_items, cap * sizeof(int4)) != cudaSuccess ||
            cudaMalloc(&h->p_cnt, need_cnt * sizeof(int)) != cudaSuccess ||
            cudaMalloc(&h->p_ctl, 4 * sizeof(int)) != cudaSuccess)
            return WF_ENOMEM;
        h->p_items_cap = cap;
        h->p_cnt_cap = need_cnt;
        drop_graphs(h);  // captured graphs hold the old buffers
    }
    std::vector<int4> items(cap);
    int counts[2] = {0, 0};  // items, items of one slot
    counts[0] = persist_items(plan, act.data(), (int)act.size(), persist_group(h), items.data(), (int)cap, &counts[1]);
    if ((size_t)counts[0] > cap) return WF_ECUDA;
    WF_TRY(cudaMemcpyAsync(h->p_items, items.data(), sizeof(int4) * std::max(counts[0], 1), cudaMemcpyHostToDevice,
                           h->stream));
    WF_TRY(cudaMemcpyAsync(h->p_ctl + 2, counts, sizeof(counts), cudaMemcpyHostToDevice, h->stream));
    WF_TRY(cudaStreamSynchronize(h->stream));  // the host vectors go out of scope
    h->p_dirty = false;
    return WF_OK;
}

cudaError_t enqueue_step(wf_handle* h) {
    const bool persistent = h->prm.scheme == WF_PR && use_persist(h) && h->p_ctl;
    cudaError_t e = enqueue_step_body(h);
    if (e == cudaSuccess && h->mms_on) e = launch_advance_time(h->tdev, h->dt, h->stream);
    // step budgets: the persistent kernel spends them itself when a slot's last item ends
    if (e == cudaSuccess && h->budget_on && !persistent) {
        const int z0 = h->gn > 0 ? h->gz0 : 0, n = h->gn > 0 ? h->gn : h->S;
        e = launch_step_budget(h->active_dev + z0, h->budget_dev + z0, n, h->stream);
    }
    return e;
}

// Point the handle's per-slot pointers (fields, flags, operators, factors, wind factors) at slot
// z0's block: launches then treat slot z0 as their first slot.  z0 = 0 restores the layout.
void rebase_slots(wf_handle* h, int z0) {
    Arena B;
    B.base = h->slots_mem + (size_t)h->sbytes * z0;
    layout_slot(h, B);
}

// Step form 3 applies to a batch of two or more slots whose steps run eagerly or from graphs
// (profiled steps and the allocation-free call take the per-pass launches).
bool use_groups(const wf_handle* h) {
    return h->tune[6] == 3 && h->S >= 2 && !h->profiling && !h->noalloc_run && !h->mms_on && h->gs;
}

// n steps of every active slot.  Step form 3: the slots are split into two groups, A (the first
// half) on the handle's stream and B on the second stream; B's quadrature of a step waits for
// A's quadrature of that step, so each group's quadrature (bound by instruction issue) runs
// beside the other group's line passes (bound by memory latency), and the two groups stay half
// a step apart until the join at the end of the n steps.  The slots are independent, so the
// results are those of the per-pass form bit for bit.
cudaError_t enqueue_steps(wf_handle* h, int n) {
    if (!use_groups(h)) {
        cudaError_t e = cudaSuccess;
        for (int k = 0; k < n && e == cudaSuccess; ++k) e = enqueue_step(h);
        return e;
    }
    const int nA = (h->S + 1) / 2;
    cudaStream_t s = h->stream, s2 = h->gs;
    cudaError_t e = cudaEventRecord(h->ev_g, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s2, h->ev_g, 0);
    for (int k = 0; k < n && e == cudaSuccess; ++k) {
        h->gz0 = 0;
        h->gn = nA;
        h->ev_rhs = h->ev_q;
        e = enqueue_step(h);
        h->ev_rhs = nullptr;
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s2, h->ev_q, 0);
        h->gz0 = nA;
        h->gn = h->S - nA;
        h->stream = s2;
        rebase_slots(h, nA);
        if (e == cudaSuccess) e = enqueue_step(h);
        rebase_slots(h, 0);
        h->stream = s;
    }
    h->gz0 = h->gn = 0;
    h->ev_rhs = nullptr;
    if (e == cudaSuccess) e = cudaEventRecord(h->ev_g, s2);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, h->ev_g, 0);
    return e;
}

cudaError_t enqueue_step_body(wf_handle* h) {
    cudaStream_t s = h->stream;
    const int prec = h->prec, p = h->p;
    Op* X = h->dx.op;
    Op* Y = h->dy.op;
    const Chunks& cx = h->dx.ch;
    const Chunks& cy = h->dy.ch;
    cudaError_t e;
    if (h->prm.scheme == WF_EXPLICIT) {
        // (M^x (x) M^y)(T^{n+1} - T^n) = tau F - tau (A_x (x) M^y) T^n - tau (M^x (x) A_y) T^n
        RhsArgs r1 = rhs_args(h, h->T, nullptr, h->Phi, h->R, h->dt, X[1], Y[0], 1.0, &X[0], &Y[1], 1.0);
        auto l1 = [&] { return rhs_and_forcing(h, r1, h->R, h->dt, nullptr, 0.0); };
        if ((e = timed(h, S_RHS1, l1)) != cudaSuccess) return e;
        if (h->ev_rhs && (e = cudaEventRecord(h->ev_rhs, s)) != cudaSuccess) return e;
        LineArgs x1 = line_args(h, 1);
        add_line(x1, h->R, h->R, X[0], cx);
        add_line(x1, h->Phi, h->Phi, X[0], cx);
        if ((e = timed(h, S_X1, [&] { return launch_xsolve(prec, p, x1, s); })) != cudaSuccess) return e;
        LineArgs y1 = line_args(h, 0);
        add_line(y1, h->R, h->T, Y[0], cy, h->T);
        add_line(y1, h->Phi, h->phi, Y[0], cy, h->phi);
        y1.status = h->status;
        if ((e = timed(h, S_Y3, [&] { return launch_ysolve(prec, p, y1, s); })) != cudaSuccess) return e;
        return cudaSuccess;
    }
    if (h->prm.scheme == WF_PR && use_persist(h) && h->p_ctl) {
        // the quadrature (and forcing) as in the per-pass form, then one launch for the rest
        const double th = 0.5 * h->dt;
        RhsArgs r1 = rhs_args(h, h->T, h->F, h->Phi, h->R, th, X[1], Y[0], 1.0, &X[0], &Y[1], 1.0);
        r1.single = 1;  // the quadrature in one launch: two launches per step in all
        auto l1 = [&] { return rhs_and_forcing(h, r1, h->R, th, h->F, 1.0); };
        if ((e = timed(h, S_RHS1, l1)) != cudaSuccess) return e;
        PersistHost ph;
        persist_args(h, &ph);
        return timed(h, S_PERSIST, [&] { return persist_step(ph, nullptr, true, s); });
    }
    if (h->prm.scheme == WF_PR) {
        const double th = 0.5 * h->dt;
        const bool once = h->prm.F_timing == WF_F_ONCE;
        RhsArgs r1 = rhs_args(h, h->T, once ? h->F : nullptr, h->Phi, h->R, th, X[1], Y[0], 1.0, &X[0], &Y[1], 1.0);
        auto l1 = [&] { return rhs_and_forcing(h, r1, h->R, th, once ? h->F : nullptr, 1.0); };
        if ((e = timed(h, S_RHS1, l1)) != cudaSuccess) return e;
        if (h->ev_rhs && (e = cudaEventRecord(h->ev_rhs, s)) != cudaSuccess) return e;
        LineArgs x1 = line_args(h, 1);
        add_line(x1, h->R, h->R, X[2], cx);
        add_line(x1, h->Phi, h->Phi, X[0], cx);
        if ((e = timed(h, S_X1, [&] { return launch_xsolve(prec, p, x1, s); })) != cudaSuccess) return e;
        LineArgs y1 = line_args(h, 0);
        add_line(y1, h->R, h->T, Y[0], cy, h->T);
        if (once) add_line(y1, h->Phi, h->phi, Y[0], cy, h->phi);
        if ((e = timed(h, S_Y1, [&] { return launch_ysolve(prec, p, y1, s); })) != cudaSuccess) return e;
        bool fused = false;
        if (once && h->tune[5] != 2) {
            // substep 2 in one x pass: R = th F + (op1_x (x) M^y) T* + (M^x (x) op1_y) T*, then M^x lines
            LineArgs x2 = line_args(h, 2);
            add_line(x2, nullptr, h->R, X[0], cx);
            x2.preT = h->T;
            x2.preF = h->F;
            x2.preFscale = th;
            x2.pc1 = 1.0;
            x2.pc2 = 1.0;
            x2.pA1 = X[1].bandP;
            x2.pB1 = Y[0].bandP;
            x2.pA2 = X[0].bandP;
            x2.pB2 = Y[1].bandP;
            e = timed(h, S_X2, [&] { return launch_xsolve(prec, p, x2, s); });
            if (e == cudaSuccess) fused = true;
            else if (e != cudaErrorNotSupported) return e;
            else cudaGetLastError();
        }
        if (once && !fused) {
            MatvecArgs mv;
            mv.Nx = h->Nx;
            mv.Ny = h->Ny;
            mv.pitch = h->pitch;
            mv.T = h->T;
            mv.F = h->F;
            mv.R = h->R;
            mv.A1 = X[1].bandP;
            mv.B1 = Y[0].bandP;
            mv.A2 = X[0].bandP;
            mv.B2 = Y[1].bandP;
            mv.Fscale = th;
            mv.c1 = 1.0;
            mv.c2 = 1.0;
            mv.b = batch(h);
            if ((e = timed(h, S_MV2, [&] { return launch_matvec(prec, p, mv, s); })) != cudaSuccess) return e;
        } else if (!once) {
            RhsArgs r2 = rhs_args(h, h->T, nullptr, nullptr, h->R, th, X[1], Y[0], 1.0, &X[0], &Y[1], 1.0);
            auto l2 = [&] { return rhs_and_forcing(h, r2, h->R, th, nullptr, 0.0); };
            if ((e = timed(h, S_RHS2, l2)) != cudaSuccess) return e;
        }
        if (!fused) {
            LineArgs x2 = line_args(h, 2);
            add_line(x2, h->R, h->R, X[0], cx);
            if ((e = timed(h, S_X2, [&] { return launch_xsolve(prec, p, x2, s); })) != cudaSuccess) return e;
        }
        LineArgs y2 = line_args(h, 0);
        add_line(y2, h->R, h->T, Y[2], cy, h->T);
        if (!once) add_line(y2, h->Phi, h->phi, Y[0], cy, h->phi);
        y2.status = h->status;
        if ((e = timed(h, S_Y3, [&] { return launch_ysolve(prec, p, y2, s); })) != cudaSuccess) return e;
        return cudaSuccess;
    }
    // Strang / Crank-Nicolson
    const double half = 0.5 * h->dt;
    RhsArgs r1 = rhs_args(h, h->T, nullptr, h->Phi, h->R, half, X[1], Y[0], 2.0, nullptr, nullptr, 0.0);
    auto l1 = [&] { return rhs_and_forcing(h, r1, h->R, half, nullptr, 0.0); };
    if ((e = timed(h, S_RHS1, l1)) != cudaSuccess) return e;
    if (h->ev_rhs && (e = cudaEventRecord(h->ev_rhs, s)) != cudaSuccess) return e;
    LineArgs x1 = line_args(h, 1);
    add_line(x1, h->R, h->R, X[2], cx);
    add_line(x1, h->Phi, h->Phi, X[0], cx);
    if ((e = timed(h, S_X1, [&] { return launch_xsolve(prec, p, x1, s); })) != cudaSuccess) return e;
    LineArgs y1 = line_args(h, 0);
    add_line(y1, h->R, h->T, Y[0], cy, h->T);
    if ((e = timed(h, S_Y1, [&] { return launch_ysolve(prec, p, y1, s); })) != cudaSuccess) return e;
    LineArgs yy = line_args(h, 0);
    add_line(yy, h->T, h->T, Y[2], cy, h->T, Y[1].bandP, 2.0);
    if ((e = timed(h, S_Y2PRE, [&] { return launch_ysolve(prec, p, yy, s); })) != cudaSuccess) return e;
    RhsArgs r2 = rhs_args(h, h->T, nullptr, nullptr, h->R, half, X[1], Y[0], 2.0, nullptr, nullptr, 0.0);
    auto l2 = [&] { return rhs_and_forcing(h, r2, h->R, half, nullptr, 0.0); };
    if ((e = timed(h, S_RHS2, l2)) != cudaSuccess) return e;
    LineArgs x2 = line_args(h, 2);
    add_line(x2, h->R, h->R, X[2], cx);
    if ((e = timed(h, S_X2, [&] { return launch_xsolve(prec, p, x2, s); })) != cudaSuccess) return e;
    LineArgs y2 = line_args(h, 0);
    add_line(y2, h->R, h->T, Y[0], cy, h->T);
    add_line(y2, h->Phi, h->phi, Y[0], cy, h->phi);
    y2.status = h->status;
    if ((e = timed(h, S_Y3, [&] { return launch_ysolve(prec, p, y2, s); })) != cudaSuccess) return e;
    return cudaSuccess;
}

void drop_graphs(wf_handle* h) {
    if (h->g1) cudaGraphExecDestroy(h->g1);
    if (h->g8) cudaGraphExecDestroy(h->g8);
    h->g1 = h->g8 = nullptr;
    h->p_dirty = true;  // shapes or wind rank may have changed the persistent plan
}

cudaError_t capture(wf_handle* h, int steps, cudaGraphExec_t* out) {
    if (prepare_persist(h) != WF_OK) return cudaErrorMemoryAllocation;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) return e;
    cudaError_t le = enqueue_steps(h, steps);
    e = cudaStreamEndCapture(h->stream, &g);
    if (le != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return le;
    }
    if (e != cudaSuccess) return e;
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    return e;
}

// The kernels are launched with the largest wind rank of any slot (lower ranks have zero factors).
void refresh_wind_rank(wf_handle* h) {
    int wr = 0;
    for (const Slot& s : h->slots) wr = std::max(wr, s.wind_rank);
    if (wr != h->wr) drop_graphs(h);
    h->wr = wr;
}

void destroy(wf_handle* h) {
    if (!h) return;
    drop_graphs(h);
    if (h->bstage) cudaFree(h->bstage);
    if (h->p_items) cudaFree(h->p_items);
    if (h->p_cnt) cudaFree(h->p_cnt);
    if (h->p_ctl) cudaFree(h->p_ctl);
    for (auto& pnd : h->pending) {
        cudaEventDestroy(pnd.a);
        cudaEventDestroy(pnd.b);
    }
    for (cudaEvent_t e : h->ev_free) cudaEventDestroy(e);
    if (h->mem) cudaFree(h->mem);
    if (h->own) cudaStreamDestroy(h->own);
    if (h->aux) cudaStreamDestroy(h->aux);
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->ev_join) cudaEventDestroy(h->ev_join);
    if (h->gs) cudaStreamDestroy(h->gs);
    if (h->io_in) cudaStreamDestroy(h->io_in);
    if (h->io_out) cudaStreamDestroy(h->io_out);
    for (cudaEvent_t e : h->ev_io)
        if (e) cudaEventDestroy(e);
    if (h->ev_q) cudaEventDestroy(h->ev_q);
    if (h->ev_g) cudaEventDestroy(h->ev_g);
    delete h;
}

// Host state of one slot in or out: FP64 or FP32 host arrays [Ny][Nx], staged on the device and
// converted to or from the slot's pitched fields.  T travels on the handle's stream and the fuel on
// its second stream, so that one field's conversion overlaps the other's copy.
int set_slot_state(wf_handle* h, int slot, const void* T, const void* fuel, int host32 = 0) {
    const size_t n = (size_t)h->Nx * h->Ny, es = host32 ? sizeof(float) : sizeof(double);
    cudaStream_t s = h->stream;
    const bool two = h->aux && h->ev_fork && h->ev_join;
    cudaStream_t s2 = two ? h->aux : s;
    char* st1 = reinterpret_cast<char*>(h->stage);
    char* st2 = st1 + n * es;
    if (two) {
        WF_TRY(cudaEventRecord(h->ev_fork, s));
        WF_TRY(cudaStreamWaitEvent(s2, h->ev_fork, 0));
    }
    WF_TRY(cudaMemcpyAsync(st1, T, n * es, cudaMemcpyHostToDevice, s));
    WF_TRY(cudaMemcpyAsync(st2, fuel, n * es, cudaMemcpyHostToDevice, s2));
    WF_TRY(launch_convert_in(h->prec, st1, host32, at(h, h->T, slot), h->Nx, h->Ny, h->pitch, s));
    WF_TRY(launch_convert_in(h->prec, st2, host32, at(h, h->phi, slot), h->Nx, h->Ny, h->pitch, s2));
    if (two) {
        WF_TRY(cudaEventRecord(h->ev_join, s2));
        WF_TRY(cudaStreamWaitEvent(s, h->ev_join, 0));
    }
    WF_TRY(cudaStreamSynchronize(s));
    return WF_OK;
}

int get_slot_state(wf_handle* h, int slot, void* T, void* fuel, int host32 = 0) {
    const size_t n = (size_t)h->Nx * h->Ny, es = host32 ? sizeof(float) : sizeof(double);
    cudaStream_t s = h->stream;
    const bool two = h->aux && h->ev_fork && h->ev_join && T && fuel;
    cudaStream_t s2 = two ? h->aux : s;
    char* st1 = reinterpret_cast<char*>(h->stage);
    char* st2 = st1 + n * es;
    if (two) {
        WF_TRY(cudaEventRecord(h->ev_fork, s));
        WF_TRY(cudaStreamWaitEvent(s2, h->ev_fork, 0));
    }
    if (T) {
        WF_TRY(launch_convert_out(h->prec, at(h, h->T, slot), st1, host32, h->Nx, h->Ny, h->pitch, s));
        WF_TRY(cudaMemcpyAsync(T, st1, n * es, cudaMemcpyDeviceToHost, s));
    }
    if (fuel) {
        WF_TRY(launch_convert_out(h->prec, at(h, h->phi, slot), st2, host32, h->Nx, h->Ny, h->pitch, s2));
        WF_TRY(cudaMemcpyAsync(fuel, st2, n * es, cudaMemcpyDeviceToHost, s2));
    }
    if (two) {
        WF_TRY(cudaEventRecord(h->ev_join, s2));
        WF_TRY(cudaStreamWaitEvent(s, h->ev_join, 0));
    }
    WF_TRY(cudaStreamSynchronize(s));
    return WF_OK;
}

int set_slot_wind_factors(wf_handle* h, int slot, int rank, const double* factors) {
    cudaStream_t s = h->stream;
    const size_t es = esize(h->prec);
    const size_t qx = (size_t)kMaxRank * h->nx * h->q, qy = (size_t)kMaxRank * h->ny * h->q;
    // unused ranks hold zeros: the kernels may run with a higher rank than this slot's
    WF_TRY(cudaMemsetAsync(at(h, h->fxq, slot), 0, qx * es, s));
    WF_TRY(cudaMemsetAsync(at(h, h->gxq, slot), 0, qy * es, s));
    WF_TRY(cudaMemsetAsync(at(h, h->fyq, slot), 0, qx * es, s));
    WF_TRY(cudaMemsetAsync(at(h, h->gyq, slot), 0, qy * es, s));
    if (rank > 0) {
        const size_t nx = (size_t)rank * h->Nx, ny = (size_t)rank * h->Ny;
        WF_TRY(cudaMemcpyAsync(h->wind64, factors, 2 * (nx + ny) * sizeof(double), cudaMemcpyHostToDevice, s));
        const double* fx = h->wind64;
        const double* gx = fx + nx;
        const double* fy = gx + ny;
        const double* gy = fy + nx;
        WF_TRY(launch_factor_points(h->prec, fx, rank, h->nx, h->p, h->dx.B64, at(h, h->fxq, slot), s));
        WF_TRY(launch_factor_points(h->prec, gx, rank, h->ny, h->p, h->dy.B64, at(h, h->gxq, slot), s));
        WF_TRY(launch_factor_points(h->prec, fy, rank, h->nx, h->p, h->dx.B64, at(h, h->fyq, slot), s));
        WF_TRY(launch_factor_points(h->prec, gy, rank, h->ny, h->p, h->dy.B64, at(h, h->gyq, slot), s));
    }
    WF_TRY(cudaStreamSynchronize(s));
    h->slots[slot].wind_rank = rank;
    refresh_wind_rank(h);
    return WF_OK;
}

bool factors_finite(const double* f, size_t n) {
    for (size_t k = 0; k < n; ++k)
        if (!isfinite(f[k])) return false;
    return true;
}

}  // namespace

extern "C" {

int wf_params_default(wf_params* p) {
    if (!p) return WF_EINVAL;
    memset(p, 0, sizeof(*p));
    p->Lx = p->Ly = 100.0;
    p->cp = 1.0;
    p->rho = 1.293;
    p->kappa = 0.3;
    p->sigma = 5.67e-8;
    p->eps = 0.05;
    p->ch = 1.0;
    p->hc = -70.0;
    p->cW = 0.5;
    p->chi = 2e-2;
    p->T_amb = 300.0;
    p->T_ig = 800.0;
    p->delta_x = 3.5e-2 / 0.05;
    p->delta_z = 1.5 * 0.05;
    p->A_r = 1e-4;
    p->M_ratio = 1.0;
    p->T_a = 300.0;
    p->heat_scale = 1e4;
    p->fuel_rate = 300.0;
    p->fuel_thresh = 0.2;
    p->thresh_guard = 1e-6;
    p->scheme = WF_PR;
    p->precision = WF_FP32;
    p->F_timing = WF_F_ONCE;
    p->scale_heat_by_fuel = 0;
    return WF_OK;
}

namespace {

bool create_args_ok(int nx, int ny, int p, double dt, const wf_params* params, int capacity) {
    if (!params || nx < 1 || ny < 1 || p < 1 || p > kMaxP || !(dt > 0.0) || !isfinite(dt)) return false;
    if (nx > (1 << 15) || ny > (1 << 15) || capacity < 1 || capacity > 65535) return false;
    return params_ok(*params);
}

// Chunk lengths tried at creation, shortest first: the truncated reduced system must neglect spike
// entries below 1e-8 (FP32) or 1e-15 (FP64), and the shortest length that does is kept.
constexpr int kBaseTries = 10;
const int kBases32[kBaseTries] = {32, 48, 64, 96, 128, 256, 512, 1024, 2048, 8192};
const int kBases64[kBaseTries] = {48, 64, 96, 128, 192, 256, 512, 1024, 2048, 8192};

// Chunks of both directions for creation attempt `attempt`: at most 32 chunks per line (one warp
// lane or one thread row each); odd lengths keep the 32 lanes of the x pass on distinct banks.
void set_chunks(wf_handle* h, int attempt) {
    const int* bases = h->prec == WF_FP32 ? kBases32 : kBases64;
    for (Dir* d : {&h->dx, &h->dy}) {
        int base = bases[attempt];
        const int need = (d->N + 31) / 32;
        if (base < need) base = need;
        base |= 1;
        d->ch = make_chunks(d->N, base, h->p);
    }
}

// Shared-region and per-slot byte counts of the handle's layout for its current chunks.
void layout_sizes(wf_handle* h, size_t* shared, long long* sbytes) {
    Arena A;
    layout_shared(h, A);
    *shared = (A.off + 255) & ~(size_t)255;
    Arena B;
    layout_slot(h, B);
    *sbytes = (long long)((B.off + 255) & ~(size_t)255);
}

// Host fields of a new handle (no device work).
void init_fields(wf_handle* h, int nx, int ny, int p, double dt, const wf_params* params, int capacity) {
    h->nx = nx;
    h->ny = ny;
    h->p = p;
    h->q = p + 1;
    h->Nx = nx + p;
    h->Ny = ny + p;
    h->pitch = (h->Nx + 31) / 32 * 32;
    h->prec = params->precision;
    h->dt = dt;
    h->prm = *params;
    h->phys = make_phys(*params);
    h->S = capacity;
    h->dx.n = nx;
    h->dx.N = h->Nx;
    h->dx.L = params->Lx;
    h->dx.h = params->Lx / nx;
    h->dy.n = ny;
    h->dy.N = h->Ny;
    h->dy.L = params->Ly;
    h->dy.h = params->Ly / ny;
    for (Dir* d : {&h->dx, &h->dy})
        for (int k = 0; k < 3; ++k) d->op[k].factored = (k != 1);
}

}  // namespace

int wf_batch_bytes(int nx, int ny, int p, double dt, const wf_params* params, int capacity, size_t* bytes) {
    if (!bytes || !create_args_ok(nx, ny, p, dt, params, capacity)) return WF_EINVAL;
    wf_handle h;
    init_fields(&h, nx, ny, p, dt, params, capacity);
    size_t most = 0;
    for (int attempt = 0; attempt < kBaseTries; ++attempt) {
        set_chunks(&h, attempt);
        size_t shared = 0;
        long long sb = 0;
        layout_sizes(&h, &shared, &sb);
        most = std::max(most, shared + (size_t)sb * capacity + 256);
    }
    *bytes = most;
    return WF_OK;
}

int wf_batch_create(int nx, int ny, int p, double dt, const wf_params* params, int capacity, wf_handle** out) {
    if (!out) return WF_EINVAL;
    *out = nullptr;
    if (!create_args_ok(nx, ny, p, dt, params, capacity)) return WF_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaFree(0) != cudaSuccess) return WF_ECUDA;

    wf_handle* h = new (std::nothrow) wf_handle();
    if (!h) return WF_ENOMEM;
    init_fields(h, nx, ny, p, dt, params, capacity);
    h->slots.assign(capacity, Slot());
    for (Slot& sl : h->slots) {
        sl.wind_x = params->wind_x;
        sl.wind_y = params->wind_y;
        set_slot_coeffs(h, sl);
    }
    h->active_host.assign(capacity, 0);
    if (cudaStreamCreateWithFlags(&h->own, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&h->aux, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming) != cudaSuccess ||
        cudaStreamCreateWithFlags(&h->gs, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_q, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_g, cudaEventDisableTiming) != cudaSuccess) {
        destroy(h);
        return WF_ECUDA;
    }
    h->stream = h->own;

    // Chunk length: the shortest of the tried lengths whose neglected spike entries stay below
    // the truncation tolerance (for the creation wind).
    const double tol = trunc_tol(h);
    int rc = WF_OK;
    size_t shared = 0;
    for (int attempt = 0; attempt < kBaseTries; ++attempt) {
        set_chunks(h, attempt);
        if (h->mem) {
            cudaFree(h->mem);
            h->mem = nullptr;
        }
        layout_sizes(h, &shared, &h->sbytes);
        h->mem_bytes = shared + (size_t)h->sbytes * capacity + 256;
        if (cudaMalloc(&h->mem, h->mem_bytes) != cudaSuccess) {
            destroy(h);
            return WF_ENOMEM;
        }
        Arena A2;
        A2.base = reinterpret_cast<char*>(h->mem);
        layout_shared(h, A2);
        Arena B2;
        B2.base = reinterpret_cast<char*>(h->mem) + shared;
        h->slots_mem = B2.base;
        layout_slot(h, B2);
        // every slot block starts zeroed (fields, guard flags, unused wind ranks); no budgets
        if (cudaMemsetAsync(B2.base, 0, (size_t)h->sbytes * capacity, h->stream) != cudaSuccess ||
            cudaMemsetAsync(h->budget_dev, 0xff, sizeof(int) * capacity, h->stream) != cudaSuccess) {
            rc = WF_ECUDA;
            break;
        }
        if ((rc = build_tables(h)) != WF_OK) break;
        double worst = 0.0;
        rc = build_factors(h, 0, tol, &worst);
        if (rc != WF_ETRUNC) break;
        if (h->dx.ch.C == 1 && h->dy.ch.C == 1) break;
    }
    for (int sl = 1; sl < capacity && rc == WF_OK; ++sl) {
        double worst = 0.0;
        rc = build_factors(h, sl, tol, &worst);
    }
    if (rc == WF_OK && (upload_active(h) != cudaSuccess || cudaStreamSynchronize(h->stream) != cudaSuccess))
        rc = WF_ECUDA;
    if (rc != WF_OK) {
        destroy(h);
        return rc;
    }
    *out = h;
    return WF_OK;
}

int wf_create(int nx, int ny, int p, double dt, const wf_params* params, wf_handle** out) {
    int rc = wf_batch_create(nx, ny, p, dt, params, 1, out);
    if (rc != WF_OK) return rc;
    (*out)->active_host[0] = 1;
    (*out)->slots[0].active = true;
    (*out)->active_dirty = true;
    if (upload_active(*out) != cudaSuccess) {
        destroy(*out);
        *out = nullptr;
        return WF_ECUDA;
    }
    return WF_OK;
}

int wf_set_state(wf_handle* h, const double* T, const double* fuel, size_t n) {
    if (!h || !T || !fuel || n != (size_t)h->Nx * h->Ny) return WF_EINVAL;
    return set_slot_state(h, 0, T, fuel);
}

int wf_set_state_f32(wf_handle* h, const float* T, const float* fuel, size_t n) {
    if (!h || !T || !fuel || n != (size_t)h->Nx * h->Ny) return WF_EINVAL;
    return set_slot_state(h, 0, T, fuel, 1);
}

int wf_set_wind(wf_handle* h, int rank, const double* factors) {
    if (!h || rank < 0 || rank > kMaxRank || (rank > 0 && !factors)) return WF_EINVAL;
    if (rank > 0 && !factors_finite(factors, 2 * (size_t)rank * (h->Nx + h->Ny))) return WF_EINVAL;
    return set_slot_wind_factors(h, 0, rank, factors);
}

int wf_set_mean_wind(wf_handle* h, int slot, double wind_x, double wind_y) {
    if (!h || slot < 0 || slot >= h->S || !isfinite(wind_x) || !isfinite(wind_y)) return WF_EINVAL;
    Slot& sl = h->slots[slot];
    if (sl.wind_x == wind_x && sl.wind_y == wind_y) return WF_OK;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return WF_ECUDA;  // steps in flight use the factors
    const double old_x = sl.wind_x, old_y = sl.wind_y;
    sl.wind_x = wind_x;
    sl.wind_y = wind_y;
    set_slot_coeffs(h, sl);
    double worst = 0.0;
    int rc = build_factors(h, slot, trunc_tol(h), &worst);
    if (rc != WF_OK) {
        // keep the slot usable: back to the previous wind (whose factors were valid)
        sl.wind_x = old_x;
        sl.wind_y = old_y;
        set_slot_coeffs(h, sl);
        const int rc2 = build_factors(h, slot, trunc_tol(h), &worst);
        return rc2 == WF_OK ? rc : rc2;
    }
    if (h->mms_on && slot == 0) {
        h->mms.wind_x = wind_x;
        h->mms.wind_y = wind_y;
        drop_graphs(h);  // the forcing launch carries the wind by value
    }
    return WF_OK;
}

int wf_batch_set_slot(wf_handle* h, int slot, const double* T, const double* fuel, double wind_x, double wind_y,
                      int wind_rank, const double* wind_factors) {
    if (!h || slot < 0 || slot >= h->S || !T || !fuel) return WF_EINVAL;
    if (!isfinite(wind_x) || !isfinite(wind_y) || wind_rank < 0 || wind_rank > kMaxRank) return WF_EINVAL;
    if (wind_rank > 0 && (!wind_factors || !factors_finite(wind_factors, 2 * (size_t)wind_rank * (h->Nx + h->Ny))))
        return WF_EINVAL;
    Slot& sl = h->slots[slot];
    if (sl.wind_x != wind_x || sl.wind_y != wind_y) {
        sl.wind_x = wind_x;
        sl.wind_y = wind_y;
        set_slot_coeffs(h, sl);
        double worst = 0.0;
        const int rc = build_factors(h, slot, trunc_tol(h), &worst);
        if (rc != WF_OK) return rc;
    }
    int rc = set_slot_wind_factors(h, slot, wind_rank, wind_factors);
    if (rc != WF_OK) return rc;
    rc = set_slot_state(h, slot, T, fuel);
    if (rc != WF_OK) return rc;
    if (cudaMemsetAsync(at(h, h->status, slot), 0, 4 * sizeof(int), h->stream) != cudaSuccess) return WF_ECUDA;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return WF_ECUDA;
    return WF_OK;
}

int wf_batch_get_slot(wf_handle* h, int slot, double* T, double* fuel) {
    if (!h || slot < 0 || slot >= h->S) return WF_EINVAL;
    return get_slot_state(h, slot, T, fuel);
}

// Every slot's state in or out in one call: host arrays [S][Ny][Nx] per field, one copy per field
// through a staging area allocated on the first call (kept with the handle), one conversion
// kernel per field over all slots.  T on the handle's stream, fuel on its second stream.
static int batch_states(wf_handle* h, const void* Tin, const void* Fin, void* Tout, void* Fout, size_t n,
                        int host32) {
    const size_t per = (size_t)h->Nx * h->Ny;
    if (n != per * (size_t)h->S) return WF_EINVAL;
    const size_t es = host32 ? sizeof(float) : sizeof(double);
    const size_t need = 2 * n * es;
    if (h->bstage_bytes < need) {
        if (cudaStreamSynchronize(h->stream) != cudaSuccess) return WF_ECUDA;
        if (h->bstage) cudaFree(h->bstage);
        h->bstage = nullptr;
        h->bstage_bytes = 0;
        if (cudaMalloc(&h->bstage, need) != cudaSuccess) return WF_ENOMEM;
        h->bstage_bytes = need;
    }
    char* st1 = reinterpret_cast<char*>(h->bstage);
    char* st2 = st1 + n * es;
    cudaStream_t s = h->stream;
    const bool two = h->aux && h->ev_fork && h->ev_join;
    cudaStream_t s2 = two ? h->aux : s;
    const bool in = Tin != nullptr;
    if (two) {
        WF_TRY(cudaEventRecord(h->ev_fork, s));
        WF_TRY(cudaStreamWaitEvent(s2, h->ev_fork, 0));
    }
    struct Field {
        const void* src;
        void* dst;
        void* dev;
        char* st;
        cudaStream_t st_s;
    } f[2] = {{Tin, Tout, h->T, st1, s}, {Fin, Fout, h->phi, st2, s2}};
    for (const Field& q : f) {
        if (in) {
            WF_TRY(cudaMemcpyAsync(q.st, q.src, n * es, cudaMemcpyHostToDevice, q.st_s));
            WF_TRY(launch_convert_batch(1, h->prec, q.st, host32, at(h, q.dev, 0), h->sbytes, h->S, h->Nx, h->Ny,
                                        h->pitch, q.st_s));
        } else if (q.dst) {
            WF_TRY(launch_convert_batch(0, h->prec, q.st, host32, at(h, q.dev, 0), h->sbytes, h->S, h->Nx, h->Ny,
                                        h->pitch, q.st_s));
            WF_TRY(cudaMemcpyAsync(q.dst, q.st, n * es, cudaMemcpyDeviceToHost, q.st_s));
        }
    }
    if (two) {
        WF_TRY(cudaEventRecord(h->ev_join, s2));
        WF_TRY(cudaStreamWaitEvent(s, h->ev_join, 0));
    }
    WF_TRY(cudaStreamSynchronize(s));
    return WF_OK;
}

// End-to-end run from host arrays, the slots in groups pipelined over four streams: the upload
// stream copies group g's host arrays into its part of the staging area, a compute stream (the
// handle's stream for even groups, the second group stream for odd ones) converts them into the
// slots' pitched fields, steps the group (its per-slot pointers rebased to its first slot, as in
// step form 3) and converts the results back into the staging part, and the download stream copies
// them out.  Group g's upload runs beside the steps of groups g-1 and g-2 and the downloads of
// earlier groups.
static int batch_run(wf_handle* h, const void* Tin, const void* Fin, void* Tout, void* Fout, size_t n, int steps,
                     int groups, int host32) {
    const size_t per = (size_t)h->Nx * h->Ny;
    if (!Tin || !Fin || !Tout || !Fout || n != per * (size_t)h->S || steps < 0 || groups < 1 || groups > 8)
        return WF_EINVAL;
    // (manufactured forcing advances the handle's time once per enqueued step: one group)
    const int G = h->mms_on ? 1 : std::min(groups, h->S);
    const size_t es = host32 ? sizeof(float) : sizeof(double);
    const size_t need = 2 * n * es;
    if (h->bstage_bytes < need) {
        if (cudaStreamSynchronize(h->stream) != cudaSuccess) return WF_ECUDA;
        if (h->bstage) cudaFree(h->bstage);
        h->bstage = nullptr;
        h->bstage_bytes = 0;
        if (cudaMalloc(&h->bstage, need) != cudaSuccess) return WF_ENOMEM;
        h->bstage_bytes = need;
    }
    if (!h->io_in) {
        if (cudaStreamCreateWithFlags(&h->io_in, cudaStreamNonBlocking) != cudaSuccess ||
            cudaStreamCreateWithFlags(&h->io_out, cudaStreamNonBlocking) != cudaSuccess)
            return WF_ECUDA;
        for (cudaEvent_t& e : h->ev_io)
            if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return WF_ECUDA;
    }
    if (upload_active(h) != cudaSuccess) return WF_ECUDA;
    const char* hin[2] = {static_cast<const char*>(Tin), static_cast<const char*>(Fin)};
    char* hout[2] = {static_cast<char*>(Tout), static_cast<char*>(Fout)};
    char* st[2] = {reinterpret_cast<char*>(h->bstage), reinterpret_cast<char*>(h->bstage) + n * es};
    void* dev[2] = {h->T, h->phi};
    cudaStream_t s = h->stream, sin = h->io_in, sout = h->io_out;
    cudaEvent_t* ev_in = h->ev_io;
    cudaEvent_t* ev_done = h->ev_io + 8;
    cudaEvent_t ev_start = h->ev_io[16], ev_end = h->ev_io[17];
    // compute streams: the groups alternate between the handle's stream and the second group
    // stream, so that a group's conversions and steps run beside its neighbour's (whose kernels fill
    // the other's last waves); each group's first quadrature starts after the previous group's, as
    // in step form 3
    const bool two = G >= 2 && h->gs && !h->profiling;
    cudaError_t e = cudaEventRecord(ev_start, s);  // after the handle's earlier work
    if (e == cudaSuccess) e = cudaStreamWaitEvent(sin, ev_start, 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(sout, ev_start, 0);
    if (e == cudaSuccess && two) e = cudaStreamWaitEvent(h->gs, ev_start, 0);
    for (int g = 0; g < G && e == cudaSuccess; ++g) {
        const int z0 = (int)((long)g * h->S / G), cnt = (int)((long)(g + 1) * h->S / G) - z0;
        const size_t off = (size_t)z0 * per * es, bytes = (size_t)cnt * per * es;
        cudaStream_t cs = (two && (g & 1)) ? h->gs : s;
        for (int f = 0; f < 2 && e == cudaSuccess; ++f)
            e = cudaMemcpyAsync(st[f] + off, hin[f] + off, bytes, cudaMemcpyHostToDevice, sin);
        if (e == cudaSuccess) e = cudaEventRecord(ev_in[g], sin);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ev_in[g], 0);
        for (int f = 0; f < 2 && e == cudaSuccess; ++f)
            e = launch_convert_batch(1, h->prec, st[f] + off, host32, at(h, dev[f], z0), h->sbytes, cnt, h->Nx,
                                     h->Ny, h->pitch, cs);
        if (e == cudaSuccess && steps > 0) {
            h->gz0 = z0;
            h->gn = cnt;
            h->stream = cs;
            rebase_slots(h, z0);
            for (int k = 0; k < steps && e == cudaSuccess; ++k) {
                if (two && k == 0 && g > 0) e = cudaStreamWaitEvent(cs, h->ev_q, 0);
                h->ev_rhs = (two && k == 0) ? h->ev_q : nullptr;
                if (e == cudaSuccess) e = enqueue_step(h);
                h->ev_rhs = nullptr;
            }
            rebase_slots(h, 0);
            h->stream = s;
            h->gz0 = h->gn = 0;
        }
        for (int f = 0; f < 2 && e == cudaSuccess; ++f)
            e = launch_convert_batch(0, h->prec, st[f] + off, host32, at(h, dev[f], z0), h->sbytes, cnt, h->Nx,
                                     h->Ny, h->pitch, cs);
        if (e == cudaSuccess) e = cudaEventRecord(ev_done[g], cs);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(sout, ev_done[g], 0);
        for (int f = 0; f < 2 && e == cudaSuccess; ++f)
            e = cudaMemcpyAsync(hout[f] + off, st[f] + off, bytes, cudaMemcpyDeviceToHost, sout);
    }
    if (e == cudaSuccess) e = cudaEventRecord(ev_end, sout);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev_end, 0);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e == cudaSuccess ? WF_OK : WF_ECUDA;
}

int wf_batch_run(wf_handle* h, const double* T_in, const double* fuel_in, double* T_out, double* fuel_out,
                 size_t n, int steps, int groups) {
    if (!h) return WF_EINVAL;
    return batch_run(h, T_in, fuel_in, T_out, fuel_out, n, steps, groups, 0);
}

int wf_batch_run_f32(wf_handle* h, const float* T_in, const float* fuel_in, float* T_out, float* fuel_out,
                     size_t n, int steps, int groups) {
    if (!h) return WF_EINVAL;
    return batch_run(h, T_in, fuel_in, T_out, fuel_out, n, steps, groups, 1);
}

int wf_batch_set_states(wf_handle* h, const double* T, const double* fuel, size_t n) {
    if (!h || !T || !fuel) return WF_EINVAL;
    return batch_states(h, T, fuel, nullptr, nullptr, n, 0);
}

int wf_batch_set_states_f32(wf_handle* h, const float* T, const float* fuel, size_t n) {
    if (!h || !T || !fuel) return WF_EINVAL;
    return batch_states(h, T, fuel, nullptr, nullptr, n, 1);
}

int wf_batch_get_states(wf_handle* h, double* T, double* fuel, size_t n) {
    if (!h) return WF_EINVAL;
    return batch_states(h, nullptr, nullptr, T, fuel, n, 0);
}

int wf_batch_get_states_f32(wf_handle* h, float* T, float* fuel, size_t n) {
    if (!h) return WF_EINVAL;
    return batch_states(h, nullptr, nullptr, T, fuel, n, 1);
}

int wf_batch_activate(wf_handle* h, int slot, int on) {
    if (!h || slot < 0 || slot >= h->S) return WF_EINVAL;
    const int v = on ? 1 : 0;
    if (h->active_host[slot] != v) {
        h->active_host[slot] = v;
        h->slots[slot].active = v != 0;
        h->active_dirty = true;
    }
    return WF_OK;
}

int wf_batch_status(wf_handle* h, int* status, int n) {
    if (!h || !status || n < h->S) return WF_EINVAL;
    WF_TRY(launch_gather_status(h->status, h->sbytes, h->S, h->status_out, 1, h->stream));
    WF_TRY(cudaMemcpyAsync(status, h->status_out, sizeof(int) * h->S, cudaMemcpyDeviceToHost, h->stream));
    WF_TRY(cudaStreamSynchronize(h->stream));
    return WF_OK;
}

int wf_batch_set_budget(wf_handle* h, int slot, int steps) {
    if (!h || slot < 0 || slot >= h->S) return WF_EINVAL;
    const int v = steps < 0 ? -1 : steps;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return WF_ECUDA;  // steps in flight spend budgets
    WF_TRY(cudaMemcpy(h->budget_dev + slot, &v, sizeof(int), cudaMemcpyHostToDevice));
    if (!h->budget_on) {
        h->budget_on = true;
        drop_graphs(h);  // every launch now reads and spends budgets
    }
    return WF_OK;
}

int wf_batch_capacity(const wf_handle* h) { return h ? h->S : WF_EINVAL; }

int wf_device_bytes(const wf_handle* h, size_t* bytes) {
    if (!h || !bytes) return WF_EINVAL;
    *bytes = h->mem_bytes;
    return WF_OK;
}

int wf_step(wf_handle* h, int nsteps) {
    if (!h || nsteps < 0) return WF_EINVAL;
    if (nsteps == 0) return WF_OK;
    if (upload_active(h) != cudaSuccess) return WF_ECUDA;
    if (h->profiling) {
        const int rc = prepare_persist(h);
        if (rc != WF_OK) return rc;
        for (int k = 0; k < nsteps; ++k)
            if (enqueue_step(h) != cudaSuccess) return WF_ECUDA;
        return WF_OK;
    }
    if (h->g1 && h->p_dirty && use_persist(h)) {
        // the active slots changed: new item list (same buffers, so the graphs stay valid unless
        // prepare_persist had to reallocate them)
        const int rc = prepare_persist(h);
        if (rc != WF_OK) return rc;
    }
    if (!h->g1) {
        if (capture(h, 1, &h->g1) != cudaSuccess) {
            drop_graphs(h);
            return WF_ECUDA;
        }
        if (capture(h, 8, &h->g8) != cudaSuccess) {
            drop_graphs(h);
            return WF_ECUDA;
        }
    }
    int k = 0;
    for (; k + 8 <= nsteps; k += 8)
        if (cudaGraphLaunch(h->g8, h->stream) != cudaSuccess) return WF_ECUDA;
    for (; k < nsteps; ++k)
        if (cudaGraphLaunch(h->g1, h->stream) != cudaSuccess) return WF_ECUDA;
    return WF_OK;
}

int wf_sync(wf_handle* h) {
    if (!h) return WF_EINVAL;
    std::vector<int> st(h->S, 0);
    const int rc = wf_batch_status(h, st.data(), h->S);
    if (rc != WF_OK) return rc;
    // a bounded wait that gave up leaves some lines of that launch unsolved: every slot's
    // result of the step is suspect, so the timeout outranks the per-slot guard
    for (int z = 0; z < h->S; ++z)
        if (st[z] & WF_STATUS_TIMEOUT) return WF_ETIMEOUT;
    for (int z = 0; z < h->S; ++z)
        if ((st[z] & WF_STATUS_UNSTABLE) && h->active_host[z]) return WF_EUNSTABLE;
    return WF_OK;
}

int wf_set_wait_limit(wf_handle* h, double seconds) {
    if (!h || !(seconds >= 0.0) || seconds > 60.0) return WF_EINVAL;
    const long long ns = (long long)(seconds * 1e9);
    if (ns != h->wait_ns) {
        h->wait_ns = ns;
        drop_graphs(h);  // the limit travels in the kernels' arguments
    }
    return WF_OK;
}

int wf_get_state(wf_handle* h, double* T, double* fuel, size_t n) {
    if (!h || n != (size_t)h->Nx * h->Ny) return WF_EINVAL;
    return get_slot_state(h, 0, T, fuel);
}

int wf_get_state_f32(wf_handle* h, float* T, float* fuel, size_t n) {
    if (!h || n != (size_t)h->Nx * h->Ny) return WF_EINVAL;
    return get_slot_state(h, 0, T, fuel, 1);
}

int wf_get_dims(const wf_handle* h, int* Nx, int* Ny, int* p, int* precision) {
    if (!h) return WF_EINVAL;
    if (Nx) *Nx = h->Nx;
    if (Ny) *Ny = h->Ny;
    if (p) *p = h->p;
    if (precision) *precision = h->prec;
    return WF_OK;
}

int wf_set_stream(wf_handle* h, void* stream) {
    if (!h) return WF_EINVAL;
    h->stream = stream ? reinterpret_cast<cudaStream_t>(stream) : h->own;
    return WF_OK;
}

int wf_set_profiling(wf_handle* h, int on) {
    if (!h) return WF_EINVAL;
    h->profiling = on != 0;
    return WF_OK;
}

int wf_kernel_times(wf_handle* h, double* ms, int* counts, char (*names)[48], int max_k) {
    if (!h || max_k < 0) return WF_EINVAL;
    for (auto& pnd : h->pending) {
        if (cudaEventSynchronize(pnd.b) != cudaSuccess) return WF_ECUDA;
        float t = 0.f;
        if (cudaEventElapsedTime(&t, pnd.a, pnd.b) != cudaSuccess) return WF_ECUDA;
        h->site_ms[pnd.site] += t;
        h->site_cnt[pnd.site] += 1;
        h->ev_free.push_back(pnd.a);
        h->ev_free.push_back(pnd.b);
    }
    h->pending.clear();
    for (int k = 0; k < S_NSITES && k < max_k; ++k) {
        if (ms) ms[k] = h->site_ms[k];
        if (counts) counts[k] = h->site_cnt[k];
        if (names) {
            strncpy(names[k], kSiteNames[k], 47);
            names[k][47] = 0;
        }
    }
    for (int k = 0; k < S_NSITES; ++k) {
        h->site_ms[k] = 0;
        h->site_cnt[k] = 0;
    }
    return S_NSITES;
}

// ---- autotuner ---------------------------------------------------------------------
//
// Launch shapes are chosen per handle by timing whole steps of the handle itself: the slot
// blocks are saved, every candidate runs warm-up + `reps` eager steps timed by one CUDA event
// pair, and the blocks are restored after each candidate, so the state after wf_autotune
// equals the state before it.  Value 0 of each shape is the launchers' own rule.

int wf_autotune(wf_handle* h, int reps) {
    if (!h || reps < 1 || reps > 100) return WF_EINVAL;
    bool any = false;
    for (int z = 0; z < h->S; ++z) any = any || h->active_host[z];
    if (!any) return WF_OK;
    // Coordinate search: one shape at a time, in launch order, the others held at their best
    // values; a candidate is rated by the device time of the whole step, because a shape
    // also changes what the next kernel finds in L2.  Two sweeps.  Segment heights include
    // values between the powers of two: the number of (strip, segment) work items against
    // the resident warps decides how full the last wave is.
    static const int kSeg[] = {0, 128, 96, 80, 64, 56, 48, 40, 32, 28, 24, 21, 20, 16, 12};
    static const int kLines[] = {0, 32, 16, 8, 4, 2, 1};
    static const int kRpw[] = {0, 1, 2, 4};
    static const int kFuse[] = {0, 2};
    static const int kModeAll[] = {1, 2, 3};  // per-pass, persistent, per-pass in two slot groups
    static const int kGroup[] = {0, 1, 2, 4, 8, 16, 32, 64};
    struct Axis {
        int q;
        const int* v;
        int n;
    };
    const bool pers = persist_supported(h->prec, h->p, h->wr) && h->prm.scheme == WF_PR &&
                      h->prm.F_timing == WF_F_ONCE;
    const bool grp = h->S >= 2 && !h->mms_on;
    int kMode[3], nMode = 0;
    for (int m : kModeAll)
        if (m == 1 || (m == 2 && pers) || (m == 3 && grp)) kMode[nMode++] = m;
    // the shapes first (in the per-pass form, the rule), then the step form with those shapes and
    // the persistent form's group size; the second sweep refines the shapes under the chosen form
    const Axis order[] = {{2, kSeg, (int)(sizeof(kSeg) / sizeof(int))},
                          {0, kLines, (int)(sizeof(kLines) / sizeof(int))},
                          {3, kRpw, (int)(sizeof(kRpw) / sizeof(int))},
                          {1, kLines, (int)(sizeof(kLines) / sizeof(int))},
                          {4, kLines, (int)(sizeof(kLines) / sizeof(int))},
                          {5, kFuse, (int)(sizeof(kFuse) / sizeof(int))},
                          {6, kMode, nMode > 1 ? nMode : 0},
                          {7, kGroup, pers && h->S > 1 ? (int)(sizeof(kGroup) / sizeof(int)) : 0}};
    const size_t bytes = (size_t)h->sbytes * h->S;
    void* snap = nullptr;
    // the slots' activity flags reach the device lazily (at the next step): send them now, or
    // freshly loaded slots would be timed as inactive
    if (upload_active(h) != cudaSuccess) return WF_ECUDA;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return WF_ECUDA;
    if (cudaMalloc(&snap, bytes) != cudaSuccess) return WF_ENOMEM;
    int rc = WF_OK;
    const bool was_profiling = h->profiling;
    int saved[kTune], best[kTune];
    for (int q = 0; q < kTune; ++q) saved[q] = best[q] = h->tune[q];
    if (cudaMemcpyAsync(snap, h->slots_mem, bytes, cudaMemcpyDeviceToDevice, h->stream) != cudaSuccess)
        rc = WF_ECUDA;
    // the start time of the forcing, which every step advances
    double t_start = 0.0;
    if (h->mms_on && cudaMemcpy(&t_start, h->tdev, sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
        rc = WF_ECUDA;
    drop_graphs(h);
    h->profiling = false;
    wf_kernel_times(h, nullptr, nullptr, nullptr, 0);  // discard kernel times collected so far
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    if (cudaEventCreate(&ev0) != cudaSuccess || cudaEventCreate(&ev1) != cudaSuccess) rc = WF_ECUDA;
    // device time of about reps steps (after one warm-up launch) with the shapes in h->tune,
    // replayed from a captured graph of up to four steps as wf_step runs them (several steps per
    // graph: step form 3 keeps its slot groups half a step apart within a graph), under one event
    // pair
    const int gsteps = std::min(reps, 4), glaunch = (reps + gsteps - 1) / gsteps;
    auto measure = [&](double* t) -> int {
        cudaGraphExec_t ge = nullptr;
        if (capture(h, gsteps, &ge) != cudaSuccess) return WF_ECUDA;
        int r = WF_OK;
        if (cudaGraphLaunch(ge, h->stream) != cudaSuccess || cudaEventRecord(ev0, h->stream) != cudaSuccess)
            r = WF_ECUDA;
        for (int k = 0; k < glaunch && r == WF_OK; ++k)
            if (cudaGraphLaunch(ge, h->stream) != cudaSuccess) r = WF_ECUDA;
        if (r == WF_OK && (cudaEventRecord(ev1, h->stream) != cudaSuccess || cudaEventSynchronize(ev1) != cudaSuccess))
            r = WF_ECUDA;
        float ms = 0.f;
        if (r == WF_OK && cudaEventElapsedTime(&ms, ev0, ev1) != cudaSuccess) r = WF_ECUDA;
        cudaGraphExecDestroy(ge);
        if (r != WF_OK) return r;
        *t = ms;
        if (cudaMemcpyAsync(h->slots_mem, snap, bytes, cudaMemcpyDeviceToDevice, h->stream) != cudaSuccess)
            return WF_ECUDA;
        if (h->mms_on &&
            cudaMemcpyAsync(h->tdev, &t_start, sizeof(double), cudaMemcpyHostToDevice, h->stream) != cudaSuccess)
            return WF_ECUDA;
        return WF_OK;
    };
    // Each axis is timed in three rounds, the candidates in alternating order, and a candidate
    // keeps its fastest round: a slow drift of the clocks under the sustained load (power
    // capping) then favours no position in the list.
    constexpr int kRounds = 3, kMaxCand = 16;
    for (int sweep = 0; sweep < 2 && rc == WF_OK; ++sweep)
        for (const Axis& ax : order) {
            // the persistent step's group size matters only when that form is the one kept
            if (ax.q == 7 && best[6] != 2) continue;
            double tmin[kMaxCand];
            for (int i = 0; i < ax.n; ++i) tmin[i] = 1e300;
            for (int round = 0; round < kRounds && rc == WF_OK; ++round)
                for (int n = 0; n < ax.n && rc == WF_OK; ++n) {
                    const int i = (round & 1) ? ax.n - 1 - n : n;
                    for (int q = 0; q < kTune; ++q) h->tune[q] = best[q];
                    h->tune[ax.q] = ax.v[i];
                    h->p_dirty = true;  // the persistent form's plan follows the shapes
                    double t = 0.0;
                    rc = measure(&t);
                    if (rc == WF_OK && t < tmin[i]) tmin[i] = t;
                }
            int bi = -1;
            for (int i = 0; i < ax.n; ++i)
                if (bi < 0 || tmin[i] < tmin[bi]) bi = i;
            if (bi >= 0) best[ax.q] = ax.v[bi];
        }
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) rc = WF_ECUDA;
    cudaFree(snap);
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    h->profiling = was_profiling;
    for (int q = 0; q < kTune; ++q) h->tune[q] = rc == WF_OK ? best[q] : saved[q];
    drop_graphs(h);
    return rc;
}

int wf_set_mms(wf_handle* h, const wf_mms* m) {
    if (!h) return WF_EINVAL;
    if (!m) {
        h->mms_on = false;
        drop_graphs(h);
        return WF_OK;
    }
    if (h->S != 1 || m->nmodes < 0 || m->nmodes > 4) return WF_EINVAL;
    for (int k = 0; k < m->nmodes; ++k)
        if (!isfinite(m->amp[k]) || !isfinite(m->kx[k]) || !isfinite(m->ky[k]) || !isfinite(m->lambda[k]))
            return WF_EINVAL;
    if (!isfinite(m->base) || !isfinite(m->t0)) return WF_EINVAL;
    MmsArgs& a = h->mms;
    memset(&a, 0, sizeof(a));
    a.nmodes = m->nmodes;
    for (int k = 0; k < m->nmodes; ++k) {
        a.amp[k] = m->amp[k];
        a.kx[k] = m->kx[k];
        a.ky[k] = m->ky[k];
        a.lambda[k] = m->lambda[k];
    }
    a.base = m->base;
    a.Lx = h->dx.L;
    a.Ly = h->dy.L;
    a.hx = h->dx.h;
    a.hy = h->dy.h;
    a.nx = h->nx;
    a.ny = h->ny;
    a.Nx = h->Nx;
    a.Ny = h->Ny;
    a.pitch = h->pitch;
    a.p = h->p;
    a.q = h->q;
    a.Bx = h->dx.B64;
    a.By = h->dy.B64;
    WF_TRY(cudaMemcpyAsync(a.xi, h->gxi, sizeof(double) * h->q, cudaMemcpyDeviceToHost, h->stream));
    WF_TRY(cudaMemcpyAsync(a.w, h->gw, sizeof(double) * h->q, cudaMemcpyDeviceToHost, h->stream));
    const Phys& c = h->phys;
    a.C_d = c.C_d;
    a.c_W = c.c_W;
    a.c_chi = c.c_chi;
    a.T_amb = c.T_amb;
    a.T_amb4 = c.T_amb * c.T_amb * c.T_amb * c.T_amb;
    a.c_rad = c.c_rad;
    a.C_nld = c.C_nld;
    a.wind_x = h->slots[0].wind_x;
    a.wind_y = h->slots[0].wind_y;
    a.t = h->tdev;
    const double t0 = m->t0;
    WF_TRY(cudaMemcpyAsync(h->tdev, &t0, sizeof(double), cudaMemcpyHostToDevice, h->stream));
    WF_TRY(cudaStreamSynchronize(h->stream));  // t0 and the node arrays are host locals
    h->mms_on = true;
    drop_graphs(h);
    return WF_OK;
}

int wf_get_time(wf_handle* h, double* t) {
    if (!h || !t) return WF_EINVAL;
    WF_TRY(cudaMemcpyAsync(t, h->tdev, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    WF_TRY(cudaStreamSynchronize(h->stream));
    return WF_OK;
}

int wf_launch_count(unsigned long long* n) {
    if (!n) return WF_EINVAL;
    *n = wf::g_launches.load(std::memory_order_relaxed);
    return WF_OK;
}

int wf_get_tuning(const wf_handle* h, int* shape) {
    if (!h || !shape) return WF_EINVAL;
    for (int q = 0; q < kTune; ++q) shape[q] = h->tune[q];
    return WF_OK;
}

int wf_set_tuning(wf_handle* h, const int* shape) {
    if (!h || !shape) return WF_EINVAL;
    for (int q = 0; q < kTune; ++q)
        if (shape[q] < 0 || shape[q] > (q == 5 ? 2 : (q == 6 ? 3 : 1024))) return WF_EINVAL;
    for (int q = 0; q < kTune; ++q) h->tune[q] = shape[q];
    drop_graphs(h);
    return WF_OK;
}

}  // extern "C"

// ---- allocation-free step ------------------------------------------------------------
//
// Scratch of wf_step_noalloc: the three intermediate fields of a step (F, Phi, R), each at
// most kNoallocMaxElems padded FP32 coefficients, in one array that every GPU loading
// this library holds until the process exits (6 MiB).  Host code must not hand the
// symbol itself to a kernel: on the host it names a host-side placeholder.  Its device
// address is looked up once per device with cudaGetSymbolAddress and cached.
constexpr size_t kNoallocMaxElems = size_t(1) << 19;
static __device__ __align__(256) float g_noalloc_scratch[3 * kNoallocMaxElems];

namespace {
constexpr int kNoallocMaxDevices = 64;
void* g_noalloc_addr[kNoallocMaxDevices] = {nullptr};
std::mutex g_noalloc_mu;

// Device address of the scratch array on the current device (set up on first use).
cudaError_t noalloc_scratch(float** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kNoallocMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_addr[dev] = p;
    }
    *out = static_cast<float*>(g_noalloc_addr[dev]);
    return cudaSuccess;
}
}  // namespace

extern "C" int wf_step_noalloc(wf_handle* h, void* T, void* fuel, int pitch, int nsteps) {
    if (!h || !T || !fuel || nsteps < 0) return WF_EINVAL;
    if (h->prec != WF_FP32 || h->S != 1) return WF_EINVAL;
    // the manufactured-solution forcing keeps its clock in the handle: stepping caller-owned
    // arrays would advance it for steps the handle itself never took
    if (h->mms_on) return WF_EINVAL;
    if (pitch < h->Nx) return WF_EINVAL;
    if ((size_t)pitch * (size_t)h->Ny > kNoallocMaxElems) return WF_EINVAL;
    if (nsteps == 0) return WF_OK;
    float* scratch = nullptr;
    if (noalloc_scratch(&scratch) != cudaSuccess) return WF_ECUDA;
    if (upload_active(h) != cudaSuccess) return WF_ECUDA;
    // Run the handle's own step sequence with the caller's state and the static scratch in
    // place of the handle's buffers.  Every scratch element a kernel reads was written earlier
    // in the same step, so nothing needs clearing between calls.
    void* save[5] = {h->T, h->phi, h->F, h->Phi, h->R};
    const int save_pitch = h->pitch;
    h->T = T;
    h->phi = fuel;
    h->F = scratch;
    h->Phi = scratch + kNoallocMaxElems;
    h->R = scratch + 2 * kNoallocMaxElems;
    h->pitch = pitch;
    cudaError_t e = cudaSuccess;
    h->noalloc_run = true;  // the persistent step's buffers may not exist yet: per-pass launches
    for (int k = 0; k < nsteps && e == cudaSuccess; ++k) e = enqueue_step(h);
    h->noalloc_run = false;
    h->T = save[0];
    h->phi = save[1];
    h->F = save[2];
    h->Phi = save[3];
    h->R = save[4];
    h->pitch = save_pitch;
    return e == cudaSuccess ? WF_OK : WF_ECUDA;
}

extern "C" {

void wf_destroy(wf_handle* h) { destroy(h); }

const char* wf_strerror(int code) {
    switch (code) {
        case WF_OK: return "ok";
        case WF_PENDING: return "pending: request not finished";
        case WF_EINVAL: return "invalid argument";
        case WF_ENOMEM: return "out of device memory or HBM budget";
        case WF_ESINGULAR: return "singular 1-D operator (pivot below 1e-300 ||A||)";
        case WF_EUNSTABLE: return "unstable: temperature non-finite or above 1e5 K";
        case WF_ETIMEOUT: return "bounded device wait timed out";
        case WF_ECUDA: return "CUDA runtime error";
        case WF_ETRUNC: return "chunked solve could not reach its truncation tolerance";
        case WF_ENOTFOUND: return "unknown request ticket";
    }
    return "unknown status code";
}

}  // extern "C"
