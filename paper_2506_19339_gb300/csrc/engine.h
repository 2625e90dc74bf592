// Plan builder and executor of the split-CTMRG runtime.
#pragma once

#include <atomic>
#include <condition_variable>
#include <exception>
#include <functional>
#include <mutex>
#include <memory>
#include <thread>
#include <unordered_map>
#include <stdexcept>
#include <string>
#include <vector>

#include "sctm_internal.h"

namespace sctm {

struct Error : std::runtime_error {
    sctm_status code;
    Error(sctm_status c, const std::string& m) : std::runtime_error(m), code(c) {}
};

// A strided view of FP64 device memory (rank <= kMaxRank).
constexpr int kMaxRank = 12;
struct Ten {
    double* p = nullptr;
    int nd = 0;
    int dim[kMaxRank] = {0};
    long long st[kMaxRank] = {0};
    long long numel() const {
        long long n = 1;
        for (int i = 0; i < nd; ++i) n *= dim[i];
        return n;
    }
};

Ten view(double* p, const std::vector<int>& dims);                 // contiguous row-major
Ten permute(const Ten& t, const std::vector<int>& perm);           // out axis k = t axis perm[k]

class Engine;

// Persistent host threads for the independent sub-plans of a parallel step: run(n, fn) calls
// fn(i) for i = 1 .. n-1 on the workers and fn(0) on the caller, waits for all of them and
// rethrows the first exception.  One pool per lane (the two networks' lanes run at once).
class WorkerPool {
public:
    explicit WorkerPool(int workers);
    ~WorkerPool();
    WorkerPool(const WorkerPool&) = delete;
    WorkerPool& operator=(const WorkerPool&) = delete;
    void run(int n, const std::function<void(int)>& fn);

private:
    void loop(int w);
    std::vector<std::thread> threads_;
    std::mutex m_;
    std::condition_variable start_cv_, done_cv_;
    const std::function<void(int)>* job_ = nullptr;
    int njob_ = 0, pending_ = 0;
    long long generation_ = 0;
    bool stop_ = false;
    std::vector<std::exception_ptr> errors_;
};

// One operation of a plan as the reverse mode sees it, recorded while the plan is built (the
// tape): a contraction, a projector pair (Eqs. "projector construction" / "projector
// construction 2" as one unit with its own backward), the Frobenius normalisation that ends a
// move, or the ln kappa of the local contractions.
struct TapeOp {
    enum Kind { CTR, PROJ, NORM, LNK } kind = CTR;
    std::string spec;   // CTR: einsum spec; PROJ: the cut labels
    Ten X, Y, O;        // CTR operands / output; PROJ: X = U (rho_T), Y = L (rho_B)
    // PROJ
    std::string tl, rl, rlL, Llab;  // truncated legs, remaining legs (U / L naming), L's labels
    Ten M, PB, PT;
    double *S = nullptr, *Us = nullptr, *Vcols = nullptr, *VT = nullptr, *scale = nullptr;
    int n = 0, chi = 0, kc = 0;
    bool vt = false;   // right vectors stored as V^T (gesvd) rather than as columns
    // NORM: (source, destination view) pairs
    std::vector<std::pair<Ten, Ten>> items;
    // LNK: Z00, Z10, Z01, Z11 scalars
    double* z[4] = {nullptr, nullptr, nullptr, nullptr};
};
using Tape = std::vector<TapeOp>;
struct Adjoint;  // backward plans and buffers of one network (adjoint.cu)

constexpr int kStreams = 10;  // stream 0 = the caller's stream; 1..9 run independent sub-plans
struct EvRec {
    int kind;
    long long flops;
    int e0, e1;
    int m = 0, n = 0, k = 0, nb = 0, prec = 0;  // contraction shape (timeline diagnostic)
    int variant = 0;                            // SCTM_KERNEL_* of the contraction
};

struct Step {
    int sid = 0;  // stream index
    virtual ~Step() = default;
    virtual void run(Engine& e) = 0;
};
using Plan = std::vector<std::unique_ptr<Step>>;

// One network (numerator with the PEPO O, or the norm with the identity PEPO).
struct Network {
    int D = 0, p = 0, d = 0, chi = 0;
    Ten C[4];      // stored corners C1..C4 [h, v]
    Ten T[4][3];   // stored edges T1..T4 x (ket, int, bra) [a, b, m]
    Ten A, O, B;   // site tensors (B aliases A)
    Plan move[4];  // SCTM_MOVE_LEFT, RIGHT, UP, DOWN
    Plan spectrum; // rho_eff singular values and ||dS||
    Plan local;    // Z00, Z10, Z01, Z11, ln kappa, bra environment E
    double* S_old = nullptr;
    double* dS = nullptr;     // device scalar
    double* lnk = nullptr;    // device [ln kappa, Z11]
    double* z[4] = {nullptr, nullptr, nullptr, nullptr};  // device Z00, Z10, Z01, Z11
    Ten E;                    // bra environment, layout of A
    int* svd_info = nullptr;  // one int per SVD step
    int n_svd = 0;
    // per-network, per-stream work buffers, sized after the plans are built
    double* splitk_ws[kStreams] = {nullptr};
    double* scale_ws[kStreams] = {nullptr};   // operand max-abs pass of the tensor-core form
    void* pack_x[kStreams] = {nullptr};       // packed tensor-core operands (per stream)
    void* pack_y[kStreams] = {nullptr};
    int* rexp[kStreams] = {nullptr};          // row / column exponents of the FP64 emulation
    size_t splitk_need[kStreams] = {0};
    void* svd_dwork[kStreams] = {nullptr};
    size_t svd_dbytes = 0;
    int svd_lwork = 0;                        // gesvd workspace in doubles (inside svd_dwork)
    double* svd_rwork[kStreams] = {nullptr};  // gesvd rwork
    std::vector<char> svd_hwork[kStreams];
    size_t svd_hbytes = 0;
    int svd_nmax = 1;
    std::vector<struct CtrStep*> ctr_steps;
    std::vector<struct PartialSvdStep*> psvd_steps;  // warm-started SVDs (SCTM_SVD_PARTIAL)
    int precision = SCTM_PREC_FP64;  // form of the mixed-eligible contractions (set_precision)
    double cutoff_now = 0.0;         // pseudo-inverse cutoff in use (raised for mixed forms)
    std::vector<struct SvdStep*> svd_steps;
    int method = SCTM_METHOD_SPLIT;       // SCTM_METHOD_SPLIT, _SPLIT_D2 or _REDUCED
    bool p4_half = false;                 // projector 4 from the 2x1-cell patch (SPLIT_D2)
    Plan site;                            // reduced method: the fused site tensor from A, O, A-bar
    Ten fused;                            // reduced method: a[m, m, m, m], m = D d D
    int tuned_emu = 0, tuned_total = 0;  // autotune: contractions on the emulation / eligible
    cudaGraph_t graph = nullptr;          // one captured warm iteration (moves + spectrum)
    cudaGraphExec_t graph_exec = nullptr;
    long long graph_launches = 0;         // this library's kernels in one replay
    Tape tape_move[4];               // reverse-mode records of the moves and the local plan
    Tape tape_local;
    std::unique_ptr<Adjoint> adj;    // built on the first adjoint gradient
    double adj_gcut = 1e-6;          // adjoint: kept singular values below this s_0 held fixed
    Network();
    ~Network();
};

class Engine {
public:
    Engine(cudaStream_t s, int precision, double cutoff);
    ~Engine();
    Engine(const Engine&) = delete;
    Engine& operator=(const Engine&) = delete;

    cudaStream_t stream;  // the caller's stream == lanes[0].streams[0]
    // Two lanes of streams and solver handles, so that the numerator and norm networks can be
    // driven from two host threads at once; the lane used is the calling thread's cur_lane.
    struct Lane {
        cudaStream_t streams[kStreams] = {nullptr};
        cusolverDnHandle_t solver[kStreams] = {nullptr};
        std::vector<cudaEvent_t> ev_pool[kStreams];
        size_t ev_used[kStreams] = {0};
        std::vector<struct EvRec> ev_recs[kStreams];
    };
    static constexpr int kLanes = 2;
    Lane lanes[kLanes];
    std::unique_ptr<WorkerPool> pools[kLanes];  // host workers of each lane's parallel steps
    static thread_local int cur_lane;
    Lane& lane() { return lanes[cur_lane]; }
    // Serialised execution (profiling): every step of every plan on the lane's stream 0, the
    // parallel sub-plans one after the other, so that an event pair around a launch measures that
    // launch alone.
    bool serial = false;
    // While an iteration is captured into a CUDA graph (this thread only), stream 0 of the lane is
    // replaced by a capture stream: the caller's stream may be the legacy default stream, which
    // cannot be captured.  The parallel sub-plans are then recorded from this thread.
    static thread_local bool capturing;
    cudaStream_t cap_stream[2] = {nullptr, nullptr};
    cudaStream_t strm(int sid) {
        if (serial || sid == 0) return capturing ? cap_stream[cur_lane] : lane().streams[0];
        return lane().streams[sid];
    }
    cusolverDnHandle_t solv(int sid) { return lane().solver[serial ? 0 : sid]; }
    // Capture one iteration of a network (its four moves and the convergence spectrum) on the
    // calling thread's lane into net.graph; false if the plan cannot be captured.
    bool capture_iteration(Network& net);
    // every partial SVD of the network holds a warm-start subspace (the next iteration takes the
    // warm path throughout; false in the other SVD modes)
    bool all_warm(const Network& net) const;
    cusolverDnParams_t solver_params = nullptr;
    int precision;      // SCTM_PREC_* currently set on the move plans' contractions
    double cutoff;
    // device flags: [0] a tensor-core contraction's bounded wait ran out, [1] a projector matrix
    // had non-finite entries (zeroed before the SVD)
    int* dev_err = nullptr;
    bool mixed_build = false;  // contractions built now may run in a mixed-precision form
    // Arithmetic of the move plans' mixed-eligible contractions (absorption, half patches,
    // rho_B rho_T, renormalisation); projector formation, the spectrum and the local
    // contractions stay FP64.
    void set_precision(Network& net, int prec);
    // per contraction shape, time the FP64 kernels against the FP64 emulation on the tensor cores
    // and keep the faster for SCTM_PREC_F64EMU (run at creation of an F64EMU context)
    void autotune(Network& net);
    // Smallest useful pseudo-inverse cutoff s_k/s_1 for a contraction form: below it the
    // singular values of rho_B rho_T are rounding noise of that form.
    static double cutoff_floor(int prec);
    // ||dS|| at which sctm_iterate leaves a mixed form for the FP64 polish
    static double switch_level(int prec);
    int svd_mode = SCTM_SVD_QR;
    bool jacobi_cluster = false;  // SCTM_JACOBI_CLUSTER: the Jacobi SVD on a cluster of CTAs
    bool dry = false;  // SCTM_DRYRUN=1: build plans with placeholder pointers, no CUDA calls
    int cur_stream = 0;  // stream index given to steps while a plan is being built

    // timing: events recorded around every contraction and SVD without host synchronisation,
    // harvested (summed) after each iteration
    bool profile = false;

    double ctr_ms = 0, svd_ms = 0;
    long long ctr_launches = 0, ctr_flops = 0, svd_calls = 0;
    // per contraction kernel (SCTM_KERNEL_*): event time, launches, algorithmic FLOPs, and the
    // bytes the contraction must move at least (operands read once, output written once)
    static constexpr int kKernels = 6;  // SCTM_KERNEL_F64 .. SCTM_KERNEL_CHOL
    double kern_ms[kKernels] = {0};
    long long kern_launches[kKernels] = {0}, kern_flops[kKernels] = {0},
              kern_bytes[kKernels] = {0};
    std::atomic<long long> kernel_launches{0};  // own kernels only (cuSOLVER's are not counted)
    int record(int sid);                                       // event index in pool sid
    void record_done(int sid, int kind, long long flops, int e0, const CtrLaunch* a = nullptr);
    void harvest();

    size_t bytes = 0;                              // device bytes allocated
    double* dalloc(long long n);                   // tracked, zero-filled device buffer
    int* ialloc(const std::vector<int>& host);     // tracked device copy of an int table
    Ten alloc(const std::vector<int>& dims) { return view(dalloc(prod(dims)), dims); }
    static long long prod(const std::vector<int>& dims) {
        long long n = 1;
        for (int x : dims) n *= x;
        return n;
    }

    // Contraction O = X * Y written as an einsum spec over single-character labels.  Labels
    // present in X and Y but not in the output are summed; labels of X (Y) only must appear in
    // the output.  With out == nullptr a contiguous output in the spec's order is allocated.
    // accumulate: O += X * Y (FP64 kernels only; used by the reverse mode).
    Ten ctr(Network& net, Plan& P, const std::string& spec, const Ten& X, const Ten& Y,
            const Ten* out = nullptr, const double* rowscale = nullptr,
            const double* colscale = nullptr, bool accumulate = false);
    // split-K workspace for the contractions net.ctr_steps[first..] built after finalize()
    void assign_workspace(Network& net, size_t first);

    struct PPair {
        Ten PB, PT;
    };
    // Eqs. "projector construction" / "projector construction 2": U (rho_T) and L (rho_B) share
    // the cut legs `labels`; `tl` are the truncated legs (in the order wanted for P_B / P_T).
    // Returns P_B[t..., chi] and P_T[chi, t...].
    PPair projector(Network& net, Plan& P, const Ten& U, const Ten& L, const std::string& labels,
                    const std::string& tl);

    void build_network(Network& net);
    // the reduced method (reduced.cu): fused site tensor, moves, spectrum, local contractions
    void build_reduced_network(Network& net);
    void init_reduced_env(Network& net);
    void finalize(Network& net);
    void run(Plan& P);
    void init_env(Network& net, unsigned long long seed);
    // Forget the warm-start subspaces of the partial SVDs: the next solve of each is a full one.
    void cold_svd(Network& net);
    // Independent sub-plans, each on its own stream and host thread (stream i+1 for sub[i]):
    // they start after everything already on stream 0 and stream 0 waits for all of them.
    void parallel(Plan& P, std::vector<Plan>&& sub);
    void push(Plan& P, std::unique_ptr<Step> st) {
        st->sid = cur_stream;
        P.push_back(std::move(st));
    }
    void run_sub(Plan& P);

    // ---- reverse mode (adjoint.cu)
    Tape* tape = nullptr;   // while a plan is built: where its operations are recorded
    int in_proj = 0;        // > 0 inside projector(): its contractions belong to the PROJ record
    bool force_full_svd = false;  // partial-SVD steps run their full (gesvd) solve
    long long size_of(const double* base) const;  // doubles of a dalloc'd buffer (0 if unknown)
    // d f / d A of one network's ln kappa at its converged environment, by implicit
    // differentiation of the split-CTMRG fixed point (restarted GMRES on (I - J^T) lambda = w,
    // J the Jacobian of one iteration, w = d ln kappa / d E).  dA: p D^4 device doubles (set).
    // Returns the matrix-vector products used and the final relative residual.
    void adjoint_lnk_grad(Network& net, double* dA, double tol, int max_mv, int* mv_used,
                          double* residual);
    // build the backward plans from the tapes (done by the first adjoint_lnk_grad; with
    // SCTM_DRYRUN=1 it only checks every backward contraction's labels and shapes)
    void build_adjoint(Network& net);

private:
    std::unordered_map<const double*, long long> sizes_;
    std::vector<void*> allocs_;
    std::vector<cudaEvent_t> owned_events_;
    char dry_base_[64] = {0};
};

// the convergence spectrum plan (Sec. III.D), shared by both methods
void build_spectrum(Engine& e, Network& net);

}  // namespace sctm
