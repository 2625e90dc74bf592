// Plan builder and executor of the split-CTMRG runtime.
#pragma once

#include <atomic>
#include <functional>
#include <memory>
#include <thread>
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
    static thread_local int cur_lane;
    Lane& lane() { return lanes[cur_lane]; }
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
    // Smallest useful pseudo-inverse cutoff s_k/s_1 for a contraction form: below it the
    // singular values of rho_B rho_T are rounding noise of that form.
    static double cutoff_floor(int prec);
    // ||dS|| at which sctm_iterate leaves a mixed form for the FP64 polish
    static double switch_level(int prec);
    int svd_mode = SCTM_SVD_QR;
    bool dry = false;  // SCTM_DRYRUN=1: build plans with placeholder pointers, no CUDA calls
    int cur_stream = 0;  // stream index given to steps while a plan is being built

    // timing: events recorded around every contraction and SVD without host synchronisation,
    // harvested (summed) after each iteration
    bool profile = false;

    double ctr_ms = 0, svd_ms = 0;
    long long ctr_launches = 0, ctr_flops = 0, svd_calls = 0;
    // per contraction kernel (SCTM_KERNEL_*): event time, launches, algorithmic FLOPs, and the
    // bytes the contraction must move at least (operands read once, output written once)
    double kern_ms[4] = {0, 0, 0, 0};
    long long kern_launches[4] = {0, 0, 0, 0}, kern_flops[4] = {0, 0, 0, 0},
              kern_bytes[4] = {0, 0, 0, 0};
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
    Ten ctr(Network& net, Plan& P, const std::string& spec, const Ten& X, const Ten& Y,
            const Ten* out = nullptr, const double* rowscale = nullptr,
            const double* colscale = nullptr);

    struct PPair {
        Ten PB, PT;
    };
    // Eqs. "projector construction" / "projector construction 2": U (rho_T) and L (rho_B) share
    // the cut legs `labels`; `tl` are the truncated legs (in the order wanted for P_B / P_T).
    // Returns P_B[t..., chi] and P_T[chi, t...].
    PPair projector(Network& net, Plan& P, const Ten& U, const Ten& L, const std::string& labels,
                    const std::string& tl);

    void build_network(Network& net);
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

private:
    std::vector<void*> allocs_;
    std::vector<cudaEvent_t> owned_events_;
    char dry_base_[64] = {0};
};

}  // namespace sctm
