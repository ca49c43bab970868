// Internal declarations shared by the CUDA translation units of libwf.
//
// Data layout on the device (all fields of one handle):
//   - coefficient fields T, phi, F, Phi, R: [Ny][pitch] in the handle's
//     precision P (float or double), pitch = Nx rounded up to 32 elements
//     so every row starts on a 128-byte boundary;
//   - 1-D Gauss tables per direction: B[e][a][l] = B_{e+l}(x_{e,a}) and the
//     derivative D[e][a][l], e < n, a < q = p+1, l <= p; weights w[a]*h;
//   - 1-D banded matrices: band[r][d] = A[r][r+d-p], d in [0, 2p], zero
//     outside the matrix;
//   - chunked LU factors of a 1-D operator (see Factor below).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <type_traits>

namespace wf {

constexpr int kMaxP = 3;
constexpr int kMaxRank = 4;

// Scenario batching.  Every per-scenario pointer handed to a kernel addresses scenario 0;
// scenario z's copy lies z * sbytes bytes further (each scenario owns one block of device
// memory with the same internal layout).  Launches cover all S scenarios with grid.z = S;
// a scenario whose active flag is 0, or whose step budget is spent (0), is skipped.
// Slots of one launch (its grid.z); every per-slot pointer of the launch refers to the launch's
// first slot, the next ones follow sbytes apart (a launch over a group of slots gets pointers to
// the group's first slot).
struct Batch {
    int S;
    long long sbytes;
    const int* active;  // [S] or nullptr (all active)
    const int* budget;  // [S] step budgets (negative: unlimited) or nullptr (none)
};
#ifdef __CUDACC__
template <typename T>
__device__ __forceinline__ T* scene_ptr(T* p, const Batch& b) {
    return p ? reinterpret_cast<T*>(reinterpret_cast<char*>(const_cast<typename std::remove_const<T>::type*>(p)) +
                                    (long long)blockIdx.z * b.sbytes)
             : p;
}
__device__ __forceinline__ bool scene_active(const Batch& b) {
    return (!b.active || b.active[blockIdx.z] != 0) && (!b.budget || b.budget[blockIdx.z] != 0);
}
#endif

// Normalised model coefficients (equation divided by rho*c_p).
struct Phys {
    double C_d, C_nld, c_rad, c_chi, c_W, K_ign, k_f, T_a, T_amb, T_ig, phi_min;
    int heat_by_fuel;
};

// Partition of a line of N unknowns into C chunks: chunk k starts at k*base and has
// length base, except the last one, which has length `last` in [2p, base + 2p)
// (a single chunk, C = 1, has length N).
struct Chunks {
    int N, C, base, last;
};
__host__ __device__ inline int chunk_start(const Chunks& c, int k) { return k * c.base; }
__host__ __device__ inline int chunk_len(const Chunks& c, int k) { return k < c.C - 1 ? c.base : c.last; }
__host__ __device__ inline int chunk_of(const Chunks& c, int x) {
    const int k = x / c.base;
    return k < c.C - 1 ? k : c.C - 1;
}
// Chunk and interface types of the compact factor form: 0 = first, 1 = interior, 2 = last.
__host__ __device__ inline int chunk_type(const Chunks& c, int k) { return k == 0 ? 0 : (k == c.C - 1 ? 2 : 1); }
__host__ __device__ inline int iface_type(const Chunks& c, int k) { return k == 0 ? 0 : (k == c.C - 2 ? 2 : 1); }

// Chunked LU of a banded 1-D operator A (half-bandwidth p), truncated-SPIKE form.
//   lu[r][0..p-1]  multipliers: forward row r subtracts lu[r][i-1] * y[r-i]
//   lu[r][p]       1 / U[r][r]
//   lu[r][p+j]     U[r][r+j], j = 1..p
//   spk[r][0..p-1] V (right spike of the chunk holding r), spk[r][p..2p-1] W (left spike)
//   E[k][p][p]     (I - W_{k+1}^top V_k^bottom)^{-1} for the interface between chunks k and k+1
// Every product is chunk-local: entries coupling two chunks are carried by the spikes.
//
// Compact form: with uniform open knots every interior chunk (1 .. C-2) of an operator
// has bitwise identical factors, so three chunk types suffice whatever N is:
//   luc[t][o][2p+1], spkc[t][o][2p] for o < mmax (= base + 2p), Ec[t][p][p], t in {0,1,2}.
struct FactorV {
    Chunks ch;
    const void* lu;
    const void* spk;
    const void* E;
    int compact;  // 1 if luc/spkc/Ec are valid (interior chunks verified identical)
    int mmax;
    const void* luc;
    const void* spkc;
    const void* Ec;
    // the compact factors already in the padded shared-memory layout of the line kernels
    // (fac_pad_elems elements; one bulk copy stages them), or NULL
    const void* fpad;
};

// ---- tables and factorisation (FP64, wf_tables.cu) ---------------------------------
cudaError_t launch_gauss(double* xi, double* w, int q, cudaStream_t s);
cudaError_t launch_basis(const double* xi, int q, int n, int p, double L, double* B, double* D, cudaStream_t s);
cudaError_t launch_assemble(const double* B, const double* D, const double* w, int q, int n, int p, double h,
                            double* Mb, double* Kb, double* Gb, cudaStream_t s);
// A = aM M + aK K + aG G: full band (band64) and chunked factors; diag[0] = 1.0 if a pivot was
// below 1e-300 ||A||_inf, diag[1] = largest neglected spike entry (truncation measure).
cudaError_t launch_factor(const double* Mb, const double* Kb, const double* Gb, double aM, double aK, double aG,
                          int N, int p, Chunks ch, double* band64, double* lu64, double* spk64, double* E64,
                          double* work64, double* diag, cudaStream_t s);
cudaError_t launch_to_f32(const double* src, float* dst, size_t n, cudaStream_t s);
// Compact copies of chunk types 0/1/2 (see FactorV); diag[2] = 1.0 if an interior chunk differs
// from chunk 1 bit for bit (then the compact form must not be used).
cudaError_t launch_compact(const double* lu, const double* spk, const double* E, int p, Chunks ch, int mmax,
                           double* luc, double* spkc, double* Ec, double* diag, cudaStream_t s);
// out[r][e*q+a] = sum_l B[e][a][l] coef[r][e+l]  (1-D spline factor at Gauss points)
cudaError_t launch_factor_points(int prec, const double* coef, int rank, int n, int p, const double* B,
                                 void* out, cudaStream_t s);
// host layout [Ny][Nx] in FP64 (host32 = 0) or FP32 (host32 = 1) <-> device [Ny][pitch] in the
// handle's precision (padding columns written as zeros)
cudaError_t launch_convert_in(int prec, const void* src, int host32, void* dst, int Nx, int Ny, int pitch,
                              cudaStream_t s);
cudaError_t launch_convert_out(int prec, const void* src, void* dst, int host32, int Nx, int Ny, int pitch,
                               cudaStream_t s);
// every slot at once (dir_in 1: staged host arrays [S][Ny][Nx] -> slot fields field0 + z * sbytes;
// 0: the reverse)
cudaError_t launch_convert_batch(int dir_in, int prec, const void* host_stage, int host32, void* field0,
                                 long long sbytes, int S, int Nx, int Ny, int pitch, cudaStream_t s);
cudaError_t launch_fill(int prec, void* dst, size_t n, double v, cudaStream_t s);
cudaError_t launch_gather_status(int* status0, long long sbytes, int S, int* out, int clear, cudaStream_t s);
// end of a step: every active slot with a positive budget spends one step (at zero the slot is
// skipped by every kernel until its budget is set again)
cudaError_t launch_step_budget(const int* active, int* budget, int S, cudaStream_t s);

// ---- quadrature right-hand side (wf_rhs.cu) ---------------------------------------
// Tables of an interior element along one direction (uniform open knots: every element
// p <= e < n - p has the same ones, bitwise, as the device tables), and the Gauss weights.
struct ElemTabs {
    int ok;                   // n > 2p (interior elements exist)
    double B[4][4], D[4][4];  // [Gauss point][local basis], as in the device tables
    double w[4];              // Gauss weight x element length
    double Mb[8];             // band of an interior row of the 1-D mass matrix (rows 2p .. N-1-2p)
};

struct RhsArgs {
    int nx, ny, Nx, Ny, pitch;
    const void* T;
    const void* phi;
    void* F;    // temperature load vector (optional)
    void* Phi;  // fuel increment load vector -tau k_f int(E phi B_i B_j) (optional)
    void* R;    // Rscale F + c1 (A1 (x) B1) T + c2 (A2 (x) B2) T (optional)
    const void *Bx, *Dx, *By, *Dy, *wx, *wy;
    int wind_rank;
    const void *fxq, *gxq, *fyq, *gyq;  // [rank][n*q] factor values at Gauss points
    const void *A1, *B1, *A2, *B2;      // bands along x (A) and y (B) for R; A2 may be NULL
    double Rscale, c1, c2;
    double tau;  // full time step (fuel update)
    int seg;     // element rows per segment of the streaming kernel (0: the launcher's rule)
    // second stream and fork/join events of the handle: the quadrature's boundary items run
    // there, beside its interior items (NULL: one stream)
    cudaStream_t aux;
    cudaEvent_t ev_fork, ev_join;
    int single;  // FP32: all items in one launch (no second stream)
    ElemTabs tx, ty;
    Phys phys;
    Batch b;  // per scenario: T, phi, F, Phi, R, A1, B1, A2, B2, fxq, gxq, fyq, gyq
};
cudaError_t launch_rhs(int prec, int p, const RhsArgs& a, cudaStream_t s);
// process-wide count of the time-step kernels launched (wf_launch_count)
void count_launches(int n);
// streaming form of the same computation (wf_rhs_stream.cu); cudaErrorNotSupported for
// a wind variation of rank > 2
cudaError_t launch_rhs_stream(int prec, int p, const RhsArgs& a, cudaStream_t s);
cudaError_t launch_rhs_tile(int prec, int p, const RhsArgs& a, cudaStream_t s);  // shared-memory tiles
int rhs_items_per_dof(int p);  // informational

// ---- manufactured-solution forcing (wf_mms.cu) --------------------------------------
struct MmsArgs {
    int nmodes;
    double amp[4], kx[4], ky[4], lambda[4], base;  // u* = base + sum amp (1-cos)(1-cos) exp(-lambda t)
    double Lx, Ly, hx, hy;
    int nx, ny, Nx, Ny, pitch, p, q;
    const double *Bx, *By;  // FP64 basis tables [n][q][p+1]
    double xi[8], w[8];     // Gauss nodes and weights on [0, 1]
    double C_d, c_W, c_chi, T_amb, T_amb4, c_rad, C_nld, wind_x, wind_y;
    const double* t;        // device: start time of the step being enqueued
};
// out1 += s1 * int f B_i B_j, and out2 += s2 * the same when out2 is not NULL
cudaError_t launch_forcing(int prec, const MmsArgs& a, void* out1, double s1, void* out2, double s2,
                           cudaStream_t s);
cudaError_t launch_advance_time(double* t, double dt, cudaStream_t s);

// ---- line solves and matvec (wf_solve.cu) -------------------------------------------
struct LineArgs {
    int G;       // lines per CTA of the compact-factor kernels (0: the launcher's rule; else an upper bound)
    int rpw;     // x pass: lines per warp (0: as many as the chunks allow; 1, 2: at most that many)
    int nlines;  // number of independent lines
    int pitch;   // row pitch of the fields (elements)
    int narr;    // 1 or 2 arrays (blockIdx.y)
    const void* in[2];
    void* out[2];
    FactorV f[2];
    const void* premul[2];  // y pass only: band applied along the line before the solve (or NULL)
    double prescale[2];     // y pass only: factor of that band
    const void* base[2];    // y pass only: out = base + solution (or NULL: out = solution)
    int* status;            // y pass only: guard flag for out[0] (or NULL)
    int* tstatus;           // x pass: flag word whose bit 4 records a bounded wait that gave up
    int in_dead;            // y pass: the input arrays are dead after the pass (a kernel may use them
                            // as scratch)
    long long wait_ns;      // limit of a bounded device wait (ns of %globaltimer; 0: give up at once)
    double tmax;
    Batch b;  // per scenario: in, out, factors, premul, base, status, pre*
    // x pass only, one array: when preT is set the input line is formed in the kernel as
    // R = preFscale preF + pc1 (pA1 (x) pB1) preT + pc2 (pA2 (x) pB2) preT  (in[0] unused)
    const void* preT;
    const void* preF;
    double preFscale, pc1, pc2;
    const void *pA1, *pB1, *pA2, *pB2;
};
cudaError_t launch_xsolve(int prec, int p, const LineArgs& a, cudaStream_t s);
cudaError_t launch_ysolve(int prec, int p, const LineArgs& a, cudaStream_t s);
// compact-factor form (wf_linefast.cu); returns cudaErrorNotSupported when it cannot
// take the arguments (factors not compact, more than 256 threads, shared memory)
// Raise (never lower) the dynamic shared memory a kernel may be launched with.  The limit is a
// property of the kernel, read when a launch is made; the launches captured in a graph keep the
// size each needed, so a later, smaller request for the same kernel (another pass, other launch
// shapes) must not take the limit below them.
template <typename K>
inline cudaError_t allow_dynamic_smem(K kern, size_t bytes) {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, reinterpret_cast<const void*>(kern));
    if (e != cudaSuccess) return e;
    if ((size_t)fa.maxDynamicSharedSizeBytes >= bytes) return cudaSuccess;
    return cudaFuncSetAttribute(reinterpret_cast<const void*>(kern), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)bytes);
}
cudaError_t launch_line_fast(int prec, int p, bool xdir, const LineArgs& a, cudaStream_t s);
// elements of the padded factor block of one operator (chunk rows mmax), and the kernel that
// writes it from the compact factors (luc, spkc, Ec in the working precision)
size_t fac_pad_elems(int p, int mmax);
cudaError_t launch_pad_factors(int prec, int p, int mmax, const void* luc, const void* spkc, const void* Ec,
                               void* fpad, cudaStream_t s);

// R = Fscale F + c1 (A1 (x) B1) T + c2 (A2 (x) B2) T   (A2 may be NULL)
struct MatvecArgs {
    int Nx, Ny, pitch;
    const void* T;
    const void* F;
    void* R;
    const void *A1, *B1, *A2, *B2;
    double Fscale, c1, c2;
    Batch b;  // per scenario: every pointer
};
cudaError_t launch_matvec(int prec, int p, const MatvecArgs& a, cudaStream_t s);

// ---- persistent line passes (wf_persist.cu) -----------------------------------------
// After the quadrature launch of a Peaceman-Rachford step (one F per step), one launch runs the
// step's x, y and matvec passes for every active slot, over the (pass, slot, tile) items listed
// by persist_items; the arguments are those of the per-pass launches of the same step.
struct PersistHost {
    int prec, p;
    LineArgs x1, y1, x2, y2;  // x1 and y1 with two arrays (R, Phi), x2 and y2 with one
    MatvecArgs mv;            // substep-2 right-hand side
    int xG, yG;               // x lines and y columns per tile (0: rule)
    int nslots_cap;           // slot capacity of the handle (counter blocks)
    long long wait_ns;
    int* status;              // slot-0 flag word
    const int4* items;        // device: work items in their order
    int* ctl;                 // device: [0] ticket, [1] abort flag, [2] items, [3] items per slot
    int* cnt;                 // device: nslots_cap x cstride arrival counters
    size_t cnt_cap;           // ints allocated at cnt (the launch refuses a larger plan)
    const int* active;        // device: per-slot activity flags (an inactive slot's items are skipped)
    int* budget;              // device: per-slot step budgets, or NULL (a spent budget, 0, skips too)
};
struct PersistPlan {
    int nq, nmv, nxg, nyg, narr1, cstride, ctas, seg, xG, yG;
    size_t smem;
};
bool persist_supported(int prec, int p, int wind_rank);
// plan (and, with launch, enqueue: counter reset + one kernel) of one step; cudaErrorNotSupported
// when the persistent form cannot take these arguments
cudaError_t persist_step(const PersistHost& h, PersistPlan* plan, bool launch, cudaStream_t s);
// work items of one step for the given active slots, groups of gs slots in wavefront order;
// returns the count (entries past cap are not written) and the items of one slot
int persist_items(const PersistPlan& plan, const int* slots, int nslots, int gs, int4* out, int cap,
                  int* items_per_slot);

// launch-shape helpers shared with the host driver
int line_rows_per_cta(int prec);
size_t line_smem_bytes(int prec, const Chunks& ch);

}  // namespace wf
