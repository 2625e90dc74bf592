// Plan builder and executor of the split-CTMRG runtime (Sec. III of arXiv:2506.19339).
//
// Every directional move, the convergence check and the local contractions are compiled once,
// at context creation, into a static list of steps whose buffers, gather tables and cuSOLVER
// workspaces are all allocated up front.  An iteration is then a replay of those steps on one
// stream: no allocation, no host logic beyond the loop, one device->host scalar per iteration.
#include "engine.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <functional>
#include <map>
#include <mutex>
#include <tuple>

namespace sctm {

#define CUDA_OK(x)                                                                        \
    do {                                                                                  \
        cudaError_t e_ = (x);                                                             \
        if (e_ != cudaSuccess)                                                            \
            throw Error(e_ == cudaErrorMemoryAllocation ? SCTM_ENOMEM : SCTM_ECUDA,       \
                        std::string(#x) + ": " + cudaGetErrorString(e_));                 \
    } while (0)

#define SOLVER_OK(x)                                                                      \
    do {                                                                                  \
        cusolverStatus_t s_ = (x);                                                        \
        if (s_ != CUSOLVER_STATUS_SUCCESS)                                                \
            throw Error(SCTM_ECUSOLVER, std::string(#x) + " failed: " + std::to_string(s_)); \
    } while (0)

Ten view(double* p, const std::vector<int>& dims) {
    if ((int)dims.size() > kMaxRank) throw Error(SCTM_EINVAL, "tensor rank above kMaxRank");
    Ten t;
    t.p = p;
    t.nd = (int)dims.size();
    long long s = 1;
    for (int i = t.nd - 1; i >= 0; --i) {
        t.dim[i] = dims[i];
        t.st[i] = s;
        s *= dims[i];
    }
    return t;
}

Ten permute(const Ten& t, const std::vector<int>& perm) {
    Ten o;
    o.p = t.p;
    o.nd = t.nd;
    for (int k = 0; k < t.nd; ++k) {
        o.dim[k] = t.dim[perm[k]];
        o.st[k] = t.st[perm[k]];
    }
    return o;
}

// ---------------------------------------------------------------------------------------------
// steps
// ---------------------------------------------------------------------------------------------
enum { KIND_CTR = 0, KIND_SVD = 1, KIND_FN = 2 };

struct CtrStep : Step {
    CtrLaunch a;
    size_t partial_need = 0;
    long long flops = 0;
    bool mixed_ok = false;  // may run in a tensor-core form
    bool emu_ok = false;    // SCTM_PREC_F64EMU runs it on the emulation kernel (autotune)
    void run(Engine& e) override {
        const int e0 = e.profile ? e.record(sid) : -1;
        launch_ctr(a, e.strm(sid));
        const bool tc = a.precision != SCTM_PREC_FP64;
        const int splits = tc ? a.tc_splits : (ctr_is_skinny(a) ? 1 : a.splits);
        e.kernel_launches += (splits > 1 ? 2 : 1) + (tc ? 2 : 0);
        if (e.profile) e.record_done(sid, KIND_CTR, flops, e0, &a);
    }
};

struct SvdStep : Step {
    double* M = nullptr;
    int n = 0;
    double* S = nullptr;
    double* U = nullptr;
    double* V = nullptr;  // right singular vectors: columns (polar) or rows = V^T (QR)
    bool vectors = true;
    Network* net = nullptr;
    int info_idx = 0;
    void run(Engine& e) override {
        const int e0 = e.profile ? e.record(sid) : -1;
        cusolverStatus_t st;
        if (e.svd_mode == SCTM_SVD_POLAR) {
            double herr = 0.0;
            st = cusolverDnXgesvdp(e.solv(sid), e.solver_params,
                                   vectors ? CUSOLVER_EIG_MODE_VECTOR : CUSOLVER_EIG_MODE_NOVECTOR, 1,
                                   n, n, CUDA_R_64F, M, n, CUDA_R_64F, S, CUDA_R_64F, U, n,
                                   CUDA_R_64F, V, n, CUDA_R_64F, net->svd_dwork[sid],
                                   net->svd_dbytes, net->svd_hwork[sid].data(), net->svd_hbytes,
                                   net->svd_info + info_idx, &herr);
        } else {  // gesvd writes V^T into V
            const signed char job = vectors ? 'S' : 'N';
            st = cusolverDnDgesvd(e.solv(sid), job, job, n, n, M, n, S, U, n, V, n,
                                  (double*)net->svd_dwork[sid], net->svd_lwork, net->svd_rwork[sid],
                                  net->svd_info + info_idx);
        }
        if (st != CUSOLVER_STATUS_SUCCESS)
            throw Error(SCTM_ECUSOLVER, "cuSOLVER SVD failed: " + std::to_string(st));
        if (e.profile) e.record_done(sid, KIND_SVD, 0, e0);
    }
};

// The partial SVD of one projector matrix: a full SVD (cold) while no warm-start subspace
// exists, the warm-started subspace iteration step otherwise (psvd.cu has the algorithm).
// SCTM_SVD_PARTIAL_RANDOM replaces the cold full SVD by kRandomColdSteps warm steps from a
// pseudo-random subspace (two steps meet the same parity bounds as four, at half the cold
// iteration's cost).
constexpr int kRandomColdSteps = 2;
struct PartialSvdStep : Step {
    Plan cold, warm;
    Plan seed;                // randomized cold start: a pseudo-random subspace
    bool is_warm = false;
    bool can_warm = true;     // false when the subspace exceeds the one-CTA kernels' limit
    int random_steps = 0;     // > 0: cold solve = seed + this many warm steps instead of gesvd
    void run(Engine& e) override {
        const int e0 = e.profile ? e.record(sid) : -1;
        if (e.force_full_svd) {
            e.run_sub(cold);  // full singular basis, for the adjoint's recompute
        } else if (is_warm) {
            e.run_sub(warm);
        } else if (random_steps > 0 && can_warm) {
            e.run_sub(seed);
            for (int i = 0; i < random_steps; ++i) e.run_sub(warm);
        } else {
            e.run_sub(cold);
        }
        is_warm = can_warm;
        if (e.profile) e.record_done(sid, KIND_SVD, 0, e0);
    }
};

struct FnStep : Step {
    std::function<void(cudaStream_t)> f;
    int prof = -1;  // SCTM_KERNEL_* whose profiling counters this launch feeds (-1: none)
    explicit FnStep(std::function<void(cudaStream_t)> g, int p = -1) : f(std::move(g)), prof(p) {}
    void run(Engine& e) override {
        const int e0 = (e.profile && prof >= 0) ? e.record(sid) : -1;
        f(e.strm(sid));
        e.kernel_launches += 1;
        if (e0 >= 0) {
            e.record_done(sid, KIND_FN, 0, e0);
            e.lane().ev_recs[sid].back().variant = prof;
        }
    }
};

struct ParallelStep : Step {
    std::vector<Plan> sub;
    cudaEvent_t fork_ev = nullptr;
    std::vector<cudaEvent_t> join_ev;
    void run(Engine& e) override {
        if (e.serial) {
            for (auto& p : sub) e.run_sub(p);
            return;
        }
        Engine::Lane& L = e.lane();
        const int lane = Engine::cur_lane;
        cudaEventRecord(fork_ev, e.strm(0));
        for (size_t i = 0; i < sub.size(); ++i) cudaStreamWaitEvent(L.streams[i + 1], fork_ev, 0);
        if (Engine::capturing) {  // recording a graph: the sub-plans become parallel branches
            for (auto& p : sub) e.run_sub(p);
            for (size_t i = 0; i < sub.size(); ++i) {
                cudaEventRecord(join_ev[i], L.streams[i + 1]);
                cudaStreamWaitEvent(e.strm(0), join_ev[i], 0);
            }
            return;
        }
        std::exception_ptr err;
        try {
            // the lane's persistent workers issue the sub-plans (each on its own stream)
            e.pools[lane]->run((int)sub.size(), [&](int i) {
                Engine::cur_lane = lane;
                e.run_sub(sub[i]);
            });
        } catch (...) {
            err = std::current_exception();
        }
        for (size_t i = 0; i < sub.size(); ++i) {
            cudaEventRecord(join_ev[i], L.streams[i + 1]);
            cudaStreamWaitEvent(e.strm(0), join_ev[i], 0);
        }
        if (err) std::rethrow_exception(err);
    }
};

// ---------------------------------------------------------------------------------------------
// host worker pool
// ---------------------------------------------------------------------------------------------
WorkerPool::WorkerPool(int workers) {
    for (int w = 1; w <= workers; ++w) threads_.emplace_back([this, w] { loop(w); });
}

WorkerPool::~WorkerPool() {
    {
        std::lock_guard<std::mutex> g(m_);
        stop_ = true;
    }
    start_cv_.notify_all();
    for (auto& t : threads_) t.join();
}

void WorkerPool::loop(int w) {
    long long seen = 0;
    for (;;) {
        const std::function<void(int)>* job;
        {
            std::unique_lock<std::mutex> g(m_);
            start_cv_.wait(g, [&] { return stop_ || generation_ != seen; });
            if (stop_) return;
            seen = generation_;
            if (w >= njob_) continue;
            job = job_;
        }
        std::exception_ptr err;
        try {
            (*job)(w);
        } catch (...) {
            err = std::current_exception();
        }
        std::lock_guard<std::mutex> g(m_);
        if (err && !errors_[w]) errors_[w] = err;
        if (--pending_ == 0) done_cv_.notify_all();
    }
}

void WorkerPool::run(int n, const std::function<void(int)>& fn) {
    if (n <= 0) return;
    if (n - 1 > (int)threads_.size()) throw Error(SCTM_EINVAL, "worker pool too small");
    {
        std::lock_guard<std::mutex> g(m_);
        job_ = &fn;
        njob_ = n;
        pending_ = n - 1;
        errors_.assign(n, nullptr);
        ++generation_;
    }
    start_cv_.notify_all();
    std::exception_ptr err0;
    try {
        fn(0);
    } catch (...) {
        err0 = std::current_exception();
    }
    std::unique_lock<std::mutex> g(m_);
    done_cv_.wait(g, [&] { return pending_ == 0; });
    job_ = nullptr;
    if (err0) std::rethrow_exception(err0);
    for (auto& x : errors_)
        if (x) std::rethrow_exception(x);
}

// ---------------------------------------------------------------------------------------------
// engine
// ---------------------------------------------------------------------------------------------
thread_local int Engine::cur_lane = 0;
thread_local bool Engine::capturing = false;

Engine::Engine(cudaStream_t s, int prec, double cut) : stream(s), precision(prec), cutoff(cut) {
    const char* dr = getenv("SCTM_DRYRUN");
    dry = dr && dr[0] == '1';
    dev_err = ialloc({0, 0});
    if (dry) return;
    for (int l = 0; l < kLanes; ++l) {
        Lane& L = lanes[l];
        for (int i = 0; i < kStreams; ++i) {
            if (l == 0 && i == 0)
                L.streams[i] = s;
            else
                CUDA_OK(cudaStreamCreateWithFlags(&L.streams[i], cudaStreamNonBlocking));
            SOLVER_OK(cusolverDnCreate(&L.solver[i]));
            SOLVER_OK(cusolverDnSetStream(L.solver[i], L.streams[i]));
        }
    }
    SOLVER_OK(cusolverDnCreateParams(&solver_params));
    for (int l = 0; l < kLanes; ++l) pools[l].reset(new WorkerPool(kStreams - 1));
    for (int l = 0; l < kLanes; ++l)
        CUDA_OK(cudaStreamCreateWithFlags(&cap_stream[l], cudaStreamNonBlocking));
    const char* pf = getenv("SCTM_PROFILE");
    profile = pf && pf[0] == '1';
}

Engine::~Engine() {
    for (int l = 0; l < kLanes; ++l)
        for (int i = 0; i < kStreams; ++i)
            if (lanes[l].streams[i]) cudaStreamSynchronize(lanes[l].streams[i]);
    for (int l = 0; l < kLanes; ++l)
        if (cap_stream[l]) cudaStreamDestroy(cap_stream[l]);
    for (void* p : allocs_) cudaFree(p);
    for (cudaEvent_t ev : owned_events_) cudaEventDestroy(ev);
    for (int l = 0; l < kLanes; ++l) {
        Lane& L = lanes[l];
        for (int i = 0; i < kStreams; ++i) {
            for (cudaEvent_t ev : L.ev_pool[i]) cudaEventDestroy(ev);
            if (L.solver[i]) cusolverDnDestroy(L.solver[i]);
            if (!(l == 0 && i == 0) && L.streams[i]) cudaStreamDestroy(L.streams[i]);
        }
    }
    if (solver_params) cusolverDnDestroyParams(solver_params);
}

int Engine::record(int sid) {
    Lane& L = lane();
    if (L.ev_used[sid] == L.ev_pool[sid].size()) {
        cudaEvent_t ev;
        CUDA_OK(cudaEventCreate(&ev));
        L.ev_pool[sid].push_back(ev);
    }
    const int idx = (int)L.ev_used[sid]++;
    cudaEventRecord(L.ev_pool[sid][idx], strm(sid));
    return idx;
}

void Engine::record_done(int sid, int kind, long long flops, int e0, const CtrLaunch* a) {
    const int e1 = record(sid);
    EvRec r{kind, flops, e0, e1};
    if (a) {
        r.m = a->M;
        r.n = a->N;
        r.k = a->K;
        r.nb = a->nb;
        r.prec = a->precision;
        r.variant = a->precision == SCTM_PREC_F64EMU ? SCTM_KERNEL_F64EMU
                    : a->precision != SCTM_PREC_FP64 ? SCTM_KERNEL_TC
                    : ctr_is_skinny(*a)               ? SCTM_KERNEL_SKINNY
                                                      : SCTM_KERNEL_F64;
    }
    lane().ev_recs[sid].push_back(r);
}

void Engine::harvest() {
    // SCTM_TIMELINE=<file>: also append "lane stream kind flops start_ms end_ms" per record,
    // relative to the first record of lane 0, stream 0 (a diagnostic of stream overlap)
    const char* tl = getenv("SCTM_TIMELINE");
    FILE* tf = (tl && tl[0] && lanes[0].ev_recs[0].size() > 0) ? fopen(tl, "a") : nullptr;
    cudaEvent_t ref = tf ? lanes[0].ev_pool[0][lanes[0].ev_recs[0][0].e0] : nullptr;
    for (int l = 0; l < kLanes; ++l) {
        Lane& L = lanes[l];
        for (int sid = 0; sid < kStreams; ++sid) {
            for (const EvRec& r : L.ev_recs[sid]) {
                float ms = 0;
                CUDA_OK(cudaEventSynchronize(L.ev_pool[sid][r.e1]));
                CUDA_OK(cudaEventElapsedTime(&ms, L.ev_pool[sid][r.e0], L.ev_pool[sid][r.e1]));
                if (tf) {
                    float t0 = 0, t1 = 0;
                    cudaEventSynchronize(ref);
                    cudaEventElapsedTime(&t0, ref, L.ev_pool[sid][r.e0]);
                    cudaEventElapsedTime(&t1, ref, L.ev_pool[sid][r.e1]);
                    fprintf(tf, "%d %d %d %lld %.4f %.4f %d %d %d %d %d\n", l, sid, r.kind, r.flops,
                            t0, t1, r.m, r.n, r.k, r.nb, r.prec);
                }
                if (r.kind == KIND_CTR) {
                    ctr_ms += ms;
                    ctr_launches += 1;
                    ctr_flops += r.flops;
                    kern_ms[r.variant] += ms;
                    kern_launches[r.variant] += 1;
                    kern_flops[r.variant] += r.flops;
                    kern_bytes[r.variant] +=
                        8LL * r.nb * ((long long)r.m * r.k + (long long)r.k * r.n + (long long)r.m * r.n);
                } else if (r.kind == KIND_SVD) {
                    svd_ms += ms;
                    svd_calls += 1;
                } else {
                    kern_ms[r.variant] += ms;
                    kern_launches[r.variant] += 1;
                }
            }
            L.ev_recs[sid].clear();
            L.ev_used[sid] = 0;
        }
    }
    if (tf) fclose(tf);
}

double* Engine::dalloc(long long n) {
    if (dry) return (double*)dry_base_;
    void* p = nullptr;
    CUDA_OK(cudaMalloc(&p, std::max<long long>(n, 1) * sizeof(double)));
    allocs_.push_back(p);
    bytes += std::max<long long>(n, 1) * sizeof(double);
    CUDA_OK(cudaMemset(p, 0, std::max<long long>(n, 1) * sizeof(double)));
    sizes_[(const double*)p] = std::max<long long>(n, 1);
    return (double*)p;
}

long long Engine::size_of(const double* base) const {
    auto it = sizes_.find(base);
    return it == sizes_.end() ? 0 : it->second;
}

int* Engine::ialloc(const std::vector<int>& host) {
    if (dry) return (int*)dry_base_;
    void* p = nullptr;
    size_t bytes = std::max<size_t>(host.size(), 1) * sizeof(int);
    CUDA_OK(cudaMalloc(&p, bytes));
    allocs_.push_back(p);
    this->bytes += bytes;
    if (!host.empty())
        CUDA_OK(cudaMemcpy(p, host.data(), host.size() * sizeof(int), cudaMemcpyHostToDevice));
    return (int*)p;
}

void Engine::run_sub(Plan& P) {
    for (auto& s : P) s->run(*this);
}

void Engine::parallel(Plan& P, std::vector<Plan>&& sub) {
    if ((int)sub.size() > kStreams - 1) throw Error(SCTM_EINVAL, "too many parallel sub-plans");
    auto st = std::make_unique<ParallelStep>();
    st->sub = std::move(sub);
    st->sid = 0;
    if (!dry) {
        CUDA_OK(cudaEventCreateWithFlags(&st->fork_ev, cudaEventDisableTiming));
        owned_events_.push_back(st->fork_ev);
        st->join_ev.resize(st->sub.size());
        for (auto& ev : st->join_ev) {
            CUDA_OK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
            owned_events_.push_back(ev);
        }
    }
    P.push_back(std::move(st));
}

void Engine::run(Plan& P) {
    for (auto& s : P) s->run(*this);
}



// offsets of a multi-index group (row-major over `labs`) in a tensor with per-label strides
static std::vector<int> offsets(const std::string& labs, const std::map<char, int>& dims,
                                const std::map<char, long long>& strides) {
    long long n = 1;
    for (char c : labs) n *= dims.at(c);
    std::vector<int> out((size_t)n);
    std::vector<int> idx(labs.size(), 0);
    for (long long t = 0; t < n; ++t) {
        long long off = 0;
        for (size_t i = 0; i < labs.size(); ++i) {
            auto it = strides.find(labs[i]);
            if (it != strides.end()) off += idx[i] * it->second;
        }
        if (off > 0x7fffffffLL) throw Error(SCTM_EINVAL, "tensor too large for 32-bit offsets");
        out[(size_t)t] = (int)off;
        for (int i = (int)labs.size() - 1; i >= 0; --i) {
            if (++idx[i] < dims.at(labs[i])) break;
            idx[i] = 0;
        }
    }
    return out;
}

Ten Engine::ctr(Network& net, Plan& P, const std::string& spec, const Ten& X, const Ten& Y,
                const Ten* out, const double* rowscale, const double* colscale, bool accumulate) {
    const size_t comma = spec.find(','), arrow = spec.find("->");
    if (comma == std::string::npos || arrow == std::string::npos)
        throw Error(SCTM_EINVAL, "bad contraction spec " + spec);
    const std::string xl = spec.substr(0, comma), yl = spec.substr(comma + 1, arrow - comma - 1),
                      ol = spec.substr(arrow + 2);
    if ((int)ol.size() > kMaxRank) throw Error(SCTM_EINVAL, "output rank above kMaxRank: " + spec);
    if ((int)xl.size() != X.nd || (int)yl.size() != Y.nd)
        throw Error(SCTM_EINVAL, "rank mismatch in " + spec);
    std::map<char, int> dims;
    std::map<char, long long> sx, sy, so;
    auto add = [&](const std::string& l, const Ten& t, std::map<char, long long>& s) {
        for (size_t i = 0; i < l.size(); ++i) {
            auto it = dims.find(l[i]);
            if (it != dims.end() && it->second != t.dim[i])
                throw Error(SCTM_EINVAL, std::string("dimension mismatch for label ") + l[i] +
                                             " in " + spec);
            dims[l[i]] = t.dim[i];
            if (s.count(l[i])) throw Error(SCTM_EINVAL, "repeated label in " + spec);
            s[l[i]] = t.st[i];
        }
    };
    add(xl, X, sx);
    add(yl, Y, sy);
    std::string bl, ml, nl, kl;
    for (char c : ol) {
        if (!dims.count(c)) throw Error(SCTM_EINVAL, "unknown output label in " + spec);
        const bool inx = sx.count(c), iny = sy.count(c);
        if (inx && iny) bl += c;
        else if (inx) ml += c;
        else nl += c;
    }
    for (char c : xl) {
        if (sy.count(c) && ol.find(c) == std::string::npos) kl += c;
        if (!sy.count(c) && ol.find(c) == std::string::npos)
            throw Error(SCTM_EINVAL, "label only in the first operand and not kept: " + spec);
    }
    for (char c : yl)
        if (!sx.count(c) && ol.find(c) == std::string::npos)
            throw Error(SCTM_EINVAL, "label only in the second operand and not kept: " + spec);

    Ten O;
    if (out) {
        O = *out;
        if ((int)ol.size() != O.nd) throw Error(SCTM_EINVAL, "output rank mismatch in " + spec);
        for (size_t i = 0; i < ol.size(); ++i)
            if (O.dim[i] != dims[ol[i]]) throw Error(SCTM_EINVAL, "output dims mismatch " + spec);
    } else {
        std::vector<int> od;
        for (char c : ol) od.push_back(dims[c]);
        O = alloc(od);
    }
    for (size_t i = 0; i < ol.size(); ++i) so[ol[i]] = O.st[i];

    auto st = std::make_unique<CtrStep>();
    CtrLaunch& a = st->a;
    a.X = X.p;
    a.Y = Y.p;
    a.O = O.p;
    std::vector<int> txm = offsets(ml, dims, sx), txk = offsets(kl, dims, sx),
                     tyk = offsets(kl, dims, sy), tyn = offsets(nl, dims, sy),
                     tom = offsets(ml, dims, so), ton = offsets(nl, dims, so);
    a.M = (int)txm.size();
    a.N = (int)tyn.size();
    a.K = (int)txk.size();
    a.xm = ialloc(txm);
    a.xk = ialloc(txk);
    a.yk = ialloc(tyk);
    a.yn = ialloc(tyn);
    a.om = ialloc(tom);
    a.on = ialloc(ton);
    if (!bl.empty()) {
        std::vector<int> txb = offsets(bl, dims, sx), tyb = offsets(bl, dims, sy),
                         tob = offsets(bl, dims, so);
        a.nb = (int)txb.size();
        a.xb = ialloc(txb);
        a.yb = ialloc(tyb);
        a.ob = ialloc(tob);
    }
    a.rowscale = rowscale;
    a.colscale = colscale;
    st->mixed_ok = mixed_build;
    a.precision = mixed_build ? precision : SCTM_PREC_FP64;
    a.err = dev_err;
    // FP64 kernel: 32 x 32 tiles when 64 x 64 tiles cannot fill the 152 SMs; split K when even
    // those cannot.  Tensor-core kernel: 128 x 64 tiles, split K the same way (chunks of 32).
    const long long tiles64 = (long long)((a.M + 63) / 64) * ((a.N + 63) / 64) * a.nb;
    a.tile = tiles64 < 152 ? 32 : 64;
    auto split_k = [&](long long tiles, int align, int& splits, int& kchunk) {
        splits = 1;
        kchunk = std::max(a.K, 1);
        if (tiles < 152 && a.K > 256) {
            int want = (int)std::min<long long>(std::max<long long>(304 / tiles, 1), (a.K + 127) / 128);
            want = std::max(1, std::min(want, 128));
            int kc = (a.K + want - 1) / want;
            kc = ((kc + align - 1) / align) * align;
            const int sp = (a.K + kc - 1) / kc;
            if (sp > 1) {
                splits = sp;
                kchunk = kc;
            }
        }
    };
    split_k((long long)((a.M + a.tile - 1) / a.tile) * ((a.N + a.tile - 1) / a.tile) * a.nb, 16,
            a.splits, a.kchunk);
    split_k((long long)((a.M + 127) / 128) * ((a.N + 63) / 64) * a.nb, 32, a.tc_splits,
            a.tc_kchunk);
    const int max_splits = mixed_build ? std::max(a.splits, a.tc_splits) : a.splits;
    if (max_splits > 1) st->partial_need = (size_t)a.nb * max_splits * (size_t)a.M * a.N;
    st->flops = 2LL * a.M * a.N * (long long)a.K * a.nb;
    // SCTM_PLAN_DUMP=<file>: append "d_int stream M N K nb mixed_ok spec" per contraction built
    // (a diagnostic of the plan's shape mix; works with SCTM_DRYRUN=1 on a machine without a GPU)
    if (const char* pd = getenv("SCTM_PLAN_DUMP")) {
        if (pd[0]) {
            if (FILE* fp = fopen(pd, "a")) {
                fprintf(fp, "%d %d %d %d %d %d %d %s\n", net.d, cur_stream, a.M, a.N, a.K, a.nb,
                        mixed_build ? 1 : 0, spec.c_str());
                fclose(fp);
            }
        }
    }
    a.accumulate = accumulate ? 1 : 0;
    net.ctr_steps.push_back(st.get());
    net.splitk_need[cur_stream] = std::max(net.splitk_need[cur_stream], st->partial_need);
    push(P, std::move(st));
    if (tape && !in_proj) {
        TapeOp op;
        op.kind = TapeOp::CTR;
        op.spec = spec;
        op.X = X;
        op.Y = Y;
        op.O = O;
        tape->push_back(op);
    }
    return O;
}

void Engine::assign_workspace(Network& net, size_t first) {
    size_t need = 0;
    for (size_t i = first; i < net.ctr_steps.size(); ++i)
        need = std::max(need, net.ctr_steps[i]->partial_need);
    if (need == 0) return;
    double* ws = dalloc((long long)need);
    for (size_t i = first; i < net.ctr_steps.size(); ++i)
        if (net.ctr_steps[i]->partial_need > 0) net.ctr_steps[i]->a.partial = ws;
}

Engine::PPair Engine::projector(Network& net, Plan& P, const Ten& U, const Ten& L,
                                const std::string& labels, const std::string& tl) {
    static const std::string pool = "0123456789@$%&*+=?^~|";
    const char K = '#';
    std::string rl, rlL, Llab = labels;
    int n = 1;
    std::vector<int> rdims;
    size_t next = 0;
    for (size_t i = 0; i < labels.size(); ++i) {
        if (tl.find(labels[i]) != std::string::npos) continue;
        rl += labels[i];
        rlL += pool[next];
        Llab[i] = pool[next];
        ++next;
        rdims.push_back(U.dim[i]);
        n *= U.dim[i];
    }
    const int chi = net.chi;
    if (n < chi) throw Error(SCTM_EINVAL, "projector: remaining dimension smaller than chi");
    // M[r', r] = sum_t L[t, r'] U[t, r], column-major (row r' from L, column r from U)
    if (2 * (int)rl.size() > kMaxRank) throw Error(SCTM_EINVAL, "projector rank above kMaxRank");
    Ten M;
    M.p = dalloc((long long)n * n);
    M.nd = (int)(2 * rl.size());
    {
        long long s = 1;
        for (int i = (int)rl.size() - 1; i >= 0; --i) {
            M.dim[i] = rdims[i];
            M.st[i] = s;
            s *= rdims[i];
        }
        s = n;
        for (int i = (int)rl.size() - 1; i >= 0; --i) {
            M.dim[rl.size() + i] = rdims[i];
            M.st[rl.size() + i] = s;
            s *= rdims[i];
        }
    }
    ++in_proj;  // the contractions below are the PROJ record's, not separate tape entries
    ctr(net, P, Llab + "," + labels + "->" + rlL + rl, L, U, &M);
    const bool mixed = mixed_build;
    mixed_build = false;  // the SVD and the projector formation stay FP64
    double* S = dalloc(n);
    double* Us = dalloc((long long)n * n);
    double* Vs = dalloc((long long)n * n);
    // V layout: columns (gesvdp, partial SVD) or rows = V^T (gesvd)
    const int vt = svd_mode == SCTM_SVD_QR ? 1 : 0;
    // where the full right singular basis is after a full (gesvd / gesvdp) solve, for the
    // reverse mode: V^T rows, and the columns that the sign gauge may have flipped
    double* VT_full = vt ? Vs : nullptr;
    double* V_cols = vt ? nullptr : Vs;
    int kc_full = vt ? 0 : n;
    auto make_svd = [&](double* Vout) {
        auto sv = std::make_unique<SvdStep>();
        sv->M = M.p;
        sv->n = n;
        sv->S = S;
        sv->U = Us;
        sv->V = Vout;
        sv->vectors = true;
        sv->net = &net;
        sv->info_idx = net.n_svd++;
        net.svd_nmax = std::max(net.svd_nmax, n);
        net.svd_steps.push_back(sv.get());
        return sv;
    };
    // non-finite entries would send the QR iteration of gesvd into its iteration limit: zero
    // them and flag the iteration as failed (SCTM_ENUMERIC)
    int* nonfinite = dev_err + 1;
    const long long nn = (long long)n * n;
    push(P, std::make_unique<FnStep>([=](cudaStream_t s) { launch_sanitize(M.p, nn, nonfinite, s); }));
    if (svd_mode != SCTM_SVD_PARTIAL && svd_mode != SCTM_SVD_PARTIAL_RANDOM) {
        push(P, make_svd(Vs));
    } else {
        // subspace of chi + oversampling columns (Sec. III's partial SVD); the cold solve is
        // gesvd with its V^T turned into columns, the warm one the subspace iteration step
        // oversampling chi/4 (at least 8), reduced down to 8 where that keeps the subspace
        // within the one-CTA kernels' limit (chi <= kPsvdMaxK - 8); above kPsvdSmemK columns
        // one k x k matrix of the Cholesky-QR and Jacobi kernels lives in global scratch
        const int over = std::max(8, std::min(chi / 4, kPsvdMaxK - chi));
        const int k = std::min(n, chi + over);
        auto ps = std::make_unique<PartialSvdStep>();
        ps->can_warm = k <= kPsvdMaxK;
        double* VT = dalloc((long long)n * n);
        {
            Plan& C = ps->cold;
            push(C, make_svd(VT));
            const int kc = ps->can_warm ? k : chi;
            push(C, std::make_unique<FnStep>(
                        [=](cudaStream_t s) { launch_vt_columns(VT, Vs, n, kc, s); }));
            VT_full = VT;
            V_cols = Vs;
            kc_full = kc;
        }
        if (ps->can_warm) {
            Plan& W = ps->warm;
            auto mat = [&](double* p, int rows, int cols) {
                Ten t;
                t.p = p;
                t.nd = 2;
                t.dim[0] = rows;
                t.dim[1] = cols;
                t.st[0] = 1;
                t.st[1] = rows;
                return t;
            };
            double* Yb = dalloc((long long)n * k);
            double* Q1 = dalloc((long long)n * k);
            double* Qy = dalloc((long long)n * k);
            double* Zb = dalloc((long long)n * k);
            double* Qz = dalloc((long long)n * k);
            double* G = dalloc((long long)k * k);
            double* Tm = dalloc((long long)k * k);
            double* R1 = dalloc((long long)k * k);
            double* Ur = dalloc((long long)k * k);
            double* Wr = dalloc((long long)k * k);
            const bool big = k > kPsvdSmemK;
            const int kp2 = k + (k & 1);
            double* Xg = big ? dalloc((long long)k * k) : nullptr;
            double* Vg = big ? dalloc((long long)kp2 * (kp2 + 1)) : nullptr;
            const int info_idx = net.n_svd++;
            const Network* np = &net;  // svd_info is allocated after the plans are built
            const Ten Mv = mat(M.p, n, n);  // M[r', r] at r' + r n
            const Ten Vb = mat(Vs, n, k), Ut = mat(Us, n, k);
            const Ten Gt = mat(G, k, k), Tt = mat(Tm, k, k), Wt = mat(Wr, k, k), Urt = mat(Ur, k, k);
            // shifted Cholesky QR shift for the unit-diagonal scaled Gram matrix
            const double shift = 11.0 * ((double)n * k + (double)k * (k + 1)) * 0x1.0p-53;
            // three passes of column-scaled Cholesky QR (shifted, shifted, plain): a -> b -> c -> dst
            auto cholqr3 = [&](double* a, double* b, double* c, double* dst) {
                double* from[3] = {a, b, c};
                double* to[3] = {b, c, dst};
                for (int pass = 0; pass < 3; ++pass) {
                    const Ten x = mat(from[pass], n, k), y = mat(to[pass], n, k);
                    ctr(net, W, "ac,ad->cd", x, x, &Gt);
                    const double sh = pass < 2 ? shift : 0.0;
                    push(W, std::make_unique<FnStep>(
                                [=](cudaStream_t s) { launch_chol_orth(G, k, sh, Tm, Xg, s); },
                                SCTM_KERNEL_CHOL));
                    ctr(net, W, "ac,cd->ad", x, Tt, &y);
                }
            };
            const Ten Ybt = mat(Yb, n, k), Qyt = mat(Qy, n, k), Zbt = mat(Zb, n, k),
                      Qzt = mat(Qz, n, k), Bt = mat(R1, k, k);
            ctr(net, W, "ab,bc->ac", Mv, Vb, &Ybt);   // Y = M V_prev
            cholqr3(Yb, Q1, Zb, Qy);                  // Q_y
            ctr(net, W, "ba,bc->ac", Mv, Qyt, &Zbt);  // Z = M^T Q_y
            cholqr3(Zb, Yb, Q1, Qz);                  // Q_z
            ctr(net, W, "ac,ad->cd", Zbt, Qzt, &Bt);  // B = Z^T Q_z = Q_y^T M Q_z
            const bool jc = jacobi_cluster;
            push(W, std::make_unique<FnStep>([=](cudaStream_t s) {
                launch_jacobi_svd(R1, k, S, Ur, Wr, np->svd_info + info_idx, Vg, jc, s);
            }, SCTM_KERNEL_JACOBI));
            ctr(net, W, "ac,cd->ad", Qyt, Urt, &Ut);  // U = Q_y U_B
            ctr(net, W, "ac,cd->ad", Qzt, Wt, &Vb);   // V = Q_z V_B
            const unsigned long long salt = 0x5EEDull * (unsigned long long)(info_idx + 1);
            push(W, std::make_unique<FnStep>(
                        [=](cudaStream_t s) { launch_refill(Vs, n, k, S, salt, s); }));
            if (svd_mode == SCTM_SVD_PARTIAL_RANDOM) {
                // randomized cold start: every subspace column pseudo-random, then warm steps
                ps->random_steps = kRandomColdSteps;
                const unsigned long long seed0 = 0xC01Dull * (unsigned long long)(info_idx + 1);
                push(ps->seed, std::make_unique<FnStep>([=](cudaStream_t s) {
                    launch_refill(Vs, n, k, nullptr, seed0, s);
                }));
            }
        }
        net.psvd_steps.push_back(ps.get());
        push(P, std::move(ps));
    }
    push(P, std::make_unique<FnStep>(
        [=](cudaStream_t s) { launch_signfix(Us, Vs, n, chi, vt, s); }));
    double* scale = dalloc(chi);
    const Network* np = &net;  // the cutoff is read at launch time: it follows set_precision
    push(P, std::make_unique<FnStep>(
        [=](cudaStream_t s) { launch_scalevec(S, chi, np->cutoff_now, scale, s); }));
    // Us[r', c] = Us[r' + c n]; V[r, c] = Vs[r + c n] (polar) or Vs[c + r n] (QR: V^T)
    Ten V, Uv;
    V.p = Vs;
    Uv.p = Us;
    V.nd = Uv.nd = (int)rl.size() + 1;
    {
        long long s = 1;
        for (int i = (int)rl.size() - 1; i >= 0; --i) {
            V.dim[i] = Uv.dim[i] = rdims[i];
            Uv.st[i] = s;
            V.st[i] = vt ? s * n : s;
            s *= rdims[i];
        }
        V.dim[rl.size()] = Uv.dim[rl.size()] = chi;
        Uv.st[rl.size()] = n;
        V.st[rl.size()] = vt ? 1 : n;
    }
    PPair pp;
    pp.PB = ctr(net, P, labels + "," + rl + K + "->" + tl + K, U, V, nullptr, nullptr, scale);
    pp.PT = ctr(net, P, rlL + K + "," + Llab + "->" + K + tl, Uv, L, nullptr, scale, nullptr);
    mixed_build = mixed;
    --in_proj;
    if (tape && !in_proj) {
        TapeOp op;
        op.kind = TapeOp::PROJ;
        op.spec = labels;
        op.X = U;
        op.Y = L;
        op.tl = tl;
        op.rl = rl;
        op.rlL = rlL;
        op.Llab = Llab;
        op.M = M;
        op.PB = pp.PB;
        op.PT = pp.PT;
        op.S = S;
        op.Us = Us;
        op.Vcols = V_cols;
        op.VT = VT_full;
        op.kc = kc_full;
        op.vt = vt != 0;
        op.scale = scale;
        op.n = n;
        op.chi = chi;
        tape->push_back(op);
    }
    return pp;
}

// ---------------------------------------------------------------------------------------------
// frames: the right / up / down moves are the left move in a relabelled network
// (diagonal reflection; 180-degree rotation with ket <-> bra; both)
// ---------------------------------------------------------------------------------------------
struct Frame {
    Ten C[4];
    Ten T[4][3];
    Ten A, O, B;
};

static Frame make_frame(const Network& n, int move) {
    Frame f;
    auto tr = [](const Ten& t) { return permute(t, {1, 0}); };
    auto sw = [](const Ten& t) { return permute(t, {1, 0, 2}); };
    if (move == SCTM_MOVE_LEFT) {
        for (int i = 0; i < 4; ++i) {
            f.C[i] = n.C[i];
            for (int x = 0; x < 3; ++x) f.T[i][x] = n.T[i][x];
        }
        f.A = n.A;
        f.O = n.O;
        f.B = n.B;
    } else if (move == SCTM_MOVE_UP) {
        f.C[0] = tr(n.C[0]);
        f.C[1] = tr(n.C[3]);
        f.C[2] = tr(n.C[2]);
        f.C[3] = tr(n.C[1]);
        const int tmap[4] = {3, 2, 1, 0};
        for (int i = 0; i < 4; ++i)
            for (int x = 0; x < 3; ++x) f.T[i][x] = n.T[tmap[i]][x];
        f.A = permute(n.A, {0, 2, 1, 4, 3});
        f.B = permute(n.B, {0, 2, 1, 4, 3});
        f.O = permute(n.O, {0, 1, 3, 2, 5, 4});
    } else if (move == SCTM_MOVE_RIGHT) {
        f.C[0] = n.C[2];
        f.C[1] = n.C[3];
        f.C[2] = n.C[0];
        f.C[3] = n.C[1];
        const int tmap[4] = {2, 3, 0, 1};
        for (int i = 0; i < 4; ++i)
            for (int x = 0; x < 3; ++x) f.T[i][x] = sw(n.T[tmap[i]][2 - x]);
        f.A = permute(n.B, {0, 3, 4, 1, 2});
        f.B = permute(n.A, {0, 3, 4, 1, 2});
        f.O = permute(n.O, {1, 0, 4, 5, 2, 3});
    } else {  // down = diagonal reflection of the rotated frame
        f.C[0] = tr(n.C[2]);
        f.C[1] = tr(n.C[1]);
        f.C[2] = tr(n.C[0]);
        f.C[3] = tr(n.C[3]);
        const int tmap[4] = {1, 0, 3, 2};
        for (int i = 0; i < 4; ++i)
            for (int x = 0; x < 3; ++x) f.T[i][x] = sw(n.T[tmap[i]][2 - x]);
        f.A = permute(n.B, {0, 4, 3, 2, 1});
        f.B = permute(n.A, {0, 4, 3, 2, 1});
        f.O = permute(n.O, {1, 0, 5, 4, 3, 2});
    }
    return f;
}

// The alpha cut's one-column patch halves (rho_T, rho_B) of frame g, legs (xl, A_v, O_v, B_v, xr):
// the contractions of build_left_move's one-column patches (the alpha halves pass through the
// kappa and iota ones), for another move's frame.  The directional half projector 4 takes the up
// and down moves' projector 1 from these, on the same environment as the move's own projectors.
static void alpha_halves(Engine& e, Network& net, Plan& P, const Frame& g, Ten& Ua, Ten& La) {
    auto C = [&](const char* spec, const Ten& X, const Ten& Y) { return e.ctr(net, P, spec, X, Y); };
    const Ten &C1 = g.C[0], &C2 = g.C[1], &C3 = g.C[2], &C4 = g.C[3];
    const Ten &T1k = g.T[0][0], &T1i = g.T[0][1], &T1b = g.T[0][2];
    const Ten &T2k = g.T[1][0], &T2i = g.T[1][1], &T2b = g.T[1][2];
    const Ten &T3k = g.T[2][0], &T3i = g.T[2][1], &T3b = g.T[2][2];
    const Ten &T4k = g.T[3][0], &T4i = g.T[3][1], &T4b = g.T[3][2];
    const Ten &A = g.A, &O = g.O, &B = g.B;
    Ten X = C("av,acp->vcp", C1, T1k);
    X = C("vcp,ceo->vepo", X, T1i);
    const Ten Ct1 = C("vepo,ehb->hvpob", X, T1b);            // [h, v, ua, uo, ub]
    X = C("av,acE->vcE", C4, T3k);
    X = C("vcE,cef->veEf", X, T3i);
    const Ten Ct4 = C("veEf,ehg->hvEfg", X, T3b);            // [h, v, da, do, db]
    const Ten Ctop = C("hvpob,hw->vpobw", Ct1, C2);          // [v1, ua, uo, ub, v2]
    const Ten Cbot = C("hvEfg,hw->vEfgw", Ct4, C3);          // [v4, da, do, db, v3]
    X = C("vaobw,vxl->xaoblw", Ctop, T4k);
    X = C("xaoblw,saler->xobwser", X, A);
    const Ten Uk = C("xobwser,wyr->xesoby", X, T2k);         // (xl, A.d, s, O.u, B.u, xr)
    X = C("xesoby,xXl->Xesobyl", Uk, T4i);
    X = C("Xesobyl,tsolfr->Xebyftr", X, O);
    const Ten Ui = C("Xebyftr,yYr->XeftbY", X, T2i);         // (xl, A.d, O.d, s', B.u, xr)
    X = C("xeftby,xXl->Xeftbyl", Ui, T4b);
    X = C("Xeftbyl,tblgr->Xefygr", X, B);
    Ua = C("Xefygr,yYr->XefgY", X, T2b);                     // (xl, A_v, O_v, B_v, xr)
    X = C("vefgw,xvl->xefgwl", Cbot, T4b);
    X = C("xefgwl,tblgr->xefwtbr", X, B);
    const Ten Li = C("xefwtbr,ywr->xeftby", X, T2b);
    X = C("XeftbY,xXl->xeftbYl", Li, T4i);
    X = C("xeftbYl,tsolfr->xebYsor", X, O);
    const Ten Lk = C("xebYsor,yYr->xesoby", X, T2i);
    X = C("XesobY,xXl->xesobYl", Lk, T4k);
    X = C("xesobYl,saler->xobYar", X, A);
    La = C("xobYar,yYr->xaoby", X, T2k);
}

// ---------------------------------------------------------------------------------------------
// the left move (Sec. III.B, Fig. 5; Sec. III.C and Appendix for the projectors)
// ---------------------------------------------------------------------------------------------
// sym: the D2-symmetric iteration (Sec. III.B, Eq. "Symmetry constraints" and the symmetric
// corner absorption): the same projectors and edge update, but each corner absorbs its column
// and its row at once and both of its legs are truncated by the alpha pair.
// fu, fd: the frames of the up and down moves seen from this move (directional scheme with the
// half projector 4, net.p4_half: their projector 1 renormalises the column cuts of the 2 x 1-cell
// patch; the D2 scheme has them by symmetry).
static void build_left_move(Engine& e, Network& net, Plan& P, const Frame& f, bool sym = false,
                            const Frame* fu = nullptr, const Frame* fd = nullptr) {
    auto C = [&](const char* spec, const Ten& X, const Ten& Y) { return e.ctr(net, P, spec, X, Y); };
    const Ten &C1 = f.C[0], &C2 = f.C[1], &C3 = f.C[2], &C4 = f.C[3];
    const Ten &T1k = f.T[0][0], &T1i = f.T[0][1], &T1b = f.T[0][2];
    const Ten &T2k = f.T[1][0], &T2i = f.T[1][1], &T2b = f.T[1][2];
    const Ten &T3k = f.T[2][0], &T3i = f.T[2][1], &T3b = f.T[2][2];
    const Ten &T4k = f.T[3][0], &T4i = f.T[3][1], &T4b = f.T[3][2];
    const Ten &A = f.A, &O = f.O, &B = f.B;
    Ten X;

    // insertion + absorption of one column into the corners (Fig. 5(a),(b))
    X = C("av,acp->vcp", C1, T1k);
    X = C("vcp,ceo->vepo", X, T1i);
    const Ten Ct1 = C("vepo,ehb->hvpob", X, T1b);            // [h, v, ua, uo, ub]
    X = C("egb,gw->ewb", T1b, C2);
    X = C("ceo,ewb->cwob", T1i, X);
    const Ten Ct2 = C("hcp,cwob->hwpob", T1k, X);            // [h, w, ua, uo, ub]
    X = C("av,acE->vcE", C4, T3k);
    X = C("vcE,cef->veEf", X, T3i);
    const Ten Ct4 = C("veEf,ehg->hvEfg", X, T3b);            // [h, v, da, do, db]
    X = C("egG,gw->ewG", T3b, C3);
    X = C("cef,ewG->cwfG", T3i, X);
    const Ten Ct3 = C("hcE,cwfG->hwEfG", T3k, X);            // [h, w, da, do, db]

    // one-column patches: upper / lower halves at the kappa, iota, alpha cuts
    const Ten Ctop = C("hvpob,hw->vpobw", Ct1, C2);          // [v1, ua, uo, ub, v2]
    const Ten Cbot = C("hvEfg,hw->vEfgw", Ct4, C3);          // [v4, da, do, db, v3]
    X = C("vaobw,vxl->xaoblw", Ctop, T4k);
    X = C("xaoblw,saler->xobwser", X, A);
    const Ten Uk = C("xobwser,wyr->xesoby", X, T2k);         // (xl, A.d, s, O.u, B.u, xr)
    X = C("xesoby,xXl->Xesobyl", Uk, T4i);
    X = C("Xesobyl,tsolfr->Xebyftr", X, O);
    const Ten Ui = C("Xebyftr,yYr->XeftbY", X, T2i);         // (xl, A.d, O.d, s', B.u, xr)
    X = C("xeftby,xXl->Xeftbyl", Ui, T4b);
    X = C("Xeftbyl,tblgr->Xefygr", X, B);
    const Ten Ua = C("Xefygr,yYr->XefgY", X, T2b);           // (xl, A_v, O_v, B_v, xr)
    X = C("vefgw,xvl->xefgwl", Cbot, T4b);
    X = C("xefgwl,tblgr->xefwtbr", X, B);
    const Ten Li = C("xefwtbr,ywr->xeftby", X, T2b);
    X = C("XeftbY,xXl->xeftbYl", Li, T4i);
    X = C("xeftbYl,tsolfr->xebYsor", X, O);
    const Ten Lk = C("xebYsor,yYr->xesoby", X, T2i);
    X = C("XesobY,xXl->xesobYl", Lk, T4k);
    X = C("xesobYl,saler->xobYar", X, A);
    const Ten La = C("xobYar,yYr->xaoby", X, T2k);

    // stage 1: bra-related legs of this column (P1, P2, P3) and the mirror-image pairs of the
    // opposite boundary on the ket-related legs of the next column -- six independent SVD
    // pipelines, each on its own stream.  Three more streams meanwhile build the parts of the
    // two-column (stage 2) patches that do not involve the stage-1 projectors, so that this
    // contraction work overlaps the SVD pipelines instead of following them.
    Engine::PPair pr1[6];
    Ten ULA, URA, ULAO, URAO, Q1pre, Q2pre;           // upper halves (stream 7)
    Ten LLkpre, LRkpre, LLipre, LRipre;               // lower halves, kappa and iota (stream 8)
    Ten Q4pre, Q3pre;                                 // lower halves, alpha (stream 9)
    const bool half4 = net.p4_half && (sym || (fu && fd));
    if (net.p4_half && !half4) throw Error(SCTM_EINVAL, "half projector 4 without the up/down frames");
    Engine::PPair prU, prD;  // directional half projector 4: the up / down moves' projector 1
    {
        const Ten* U[6] = {&Ua, &Ua, &Uk, &Uk, &Ui, &Ui};
        const Ten* L[6] = {&La, &La, &Lk, &Lk, &Li, &Li};
        const char* lab[6] = {"xAOBy", "xAOBy", "xesoby", "xesoby", "xeftby", "xeftby"};
        const char* tl[6] = {"xB", "yA", "xsb", "yes", "xtb", "yet"};
        std::vector<Plan> sub(9);
        for (int i = 0; i < 6; ++i) {
            if (sym && (i & 1)) continue;  // the opposite boundary's pairs follow by symmetry
            e.cur_stream = i + 1;
            pr1[i] = e.projector(net, sub[i], *U[i], *L[i], lab[i], tl[i]);
        }
        if (sym) {
            // D2 symmetry (Appendix, captions of projectors 4-6): the rotation by 180 degrees with
            // ket <-> bra puts the right column's alpha / kappa / iota cut onto this column's
            // alpha / iota / kappa cut, (xr, A_v) onto (xl, B_v), (xr, A.d, s) onto
            // (xl, B.u, s') and (xr, A.d, s') onto (xl, B.u, s); P_B and P_T trade places
            pr1[1].PB = permute(pr1[0].PT, {1, 2, 0});
            pr1[1].PT = permute(pr1[0].PB, {2, 0, 1});
            pr1[3].PB = permute(pr1[4].PT, {1, 3, 2, 0});
            pr1[3].PT = permute(pr1[4].PB, {3, 0, 2, 1});
            pr1[5].PB = permute(pr1[2].PT, {1, 3, 2, 0});
            pr1[5].PT = permute(pr1[2].PB, {3, 0, 2, 1});
        }
        {
            Plan& S = sub[6];
            e.cur_stream = 7;
            auto D = [&](const char* spec, const Ten& X1, const Ten& Y1) { return e.ctr(net, S, spec, X1, Y1); };
            ULA = D("hpobxl,splEr->hobxsEr", D("hvpob,vxl->hpobxl", Ct1, T4k), A);
            URA = D("hpobyr,splEr->hobysEl", D("hwpob,wyr->hpobyr", Ct2, T2k), A);
            ULAO = D("hobsErXL,tsoLfR->hbErXtfR", D("hobxsEr,xXL->hobsErXL", ULA, T4i), O);
            URAO = D("hobsElYR,tsoLfR->hbElYtfL", D("hobysEl,yYR->hobsElYR", URA, T2i), O);
            Q1pre = D("hbErtfRZM,tbMgS->hErfRZgS", D("hbErXtfR,XZM->hbErtfRZM", ULAO, T4b), B);
            if (!half4)  // the upper-right quarter of the 2x2-cell patch
                Q2pre = D("hbElWtfLS,tbMgS->hElWfLMg", D("hbElYtfL,YWS->hbElWtfLS", URAO, T2b), B);
            if (half4 && !sym) {  // the up move's projector 1, on this stream after the halves
                Ten Uu, Lu;
                alpha_halves(e, net, S, *fu, Uu, Lu);
                prU = e.projector(net, S, Uu, Lu, "xAOBy", "xB");
            }
        }
        {
            Plan& S = sub[7];
            e.cur_stream = 8;
            auto D = [&](const char* spec, const Ten& X1, const Ten& Y1) { return e.ctr(net, S, spec, X1, Y1); };
            Ten Y1 = D("hvEfg,Xvm->hEfgXm", Ct4, T4b);
            Y1 = D("hEfgXm,tbmgQ->hEfXtbQ", Y1, B);
            Y1 = D("hEfXtbQ,xXl->hEftbQxl", Y1, T4i);
            LLkpre = D("hEftbQxl,tsolfR->hEbQxsoR", Y1, O);
            Y1 = D("hwEfG,Ywm->hEfGYm", Ct3, T2b);
            Y1 = D("hEfGYm,tbMGm->hEfYtbM", Y1, B);
            Y1 = D("hEfYtbM,yYl->hEftbMyl", Y1, T2i);
            LRkpre = D("hEftbMyl,tsoLfl->hEbMysoL", Y1, O);
            Y1 = D("hvEfg,xvm->hEfgxm", Ct4, T4b);
            LLipre = D("hEfgxm,tbmgQ->hEfxtbQ", Y1, B);
            Y1 = D("hwEfG,ywm->hEfGym", Ct3, T2b);
            LRipre = D("hEfGym,tbMGm->hEfytbM", Y1, B);
        }
        {
            Plan& S = sub[8];
            e.cur_stream = 9;
            auto D = [&](const char* spec, const Ten& X1, const Ten& Y1) { return e.ctr(net, S, spec, X1, Y1); };
            Ten Y1 = D("hvEfg,YvM->hEfgYM", Ct4, T4b);
            Y1 = D("hEfgYM,tbMgS->hEfYtbS", Y1, B);
            Y1 = D("hEfYtbS,XYL->hEftbSXL", Y1, T4i);
            Y1 = D("hEftbSXL,tsoLfR->hEbSXsoR", Y1, O);
            Y1 = D("hEbSXsoR,xXl->hEbSsoRxl", Y1, T4k);
            Q4pre = D("hEbSsoRxl,splEr->hbSoRxpr", Y1, A);
        }
        if (!half4) {  // the lower-right quarter of the 2x2-cell patch
            Plan& S = sub[8];
            e.cur_stream = 9;
            auto D = [&](const char* spec, const Ten& X1, const Ten& Y1) { return e.ctr(net, S, spec, X1, Y1); };
            Ten Y1 = D("hwEfg,WwS->hEfgWS", Ct3, T2b);
            Y1 = D("hEfgWS,tbMgS->hEfWtbM", Y1, B);
            Y1 = D("hEfWtbM,ZWR->hEftbMZR", Y1, T2i);
            Y1 = D("hEftbMZR,tsoLfR->hEbMZsoL", Y1, O);
            Y1 = D("hEbMZsoL,yZr->hEbMsoLyr", Y1, T2k);
            Q3pre = D("hEbMsoLyr,splEr->hbMoLypl", Y1, A);
        }
        if (half4 && !sym) {  // the down move's projector 1
            Plan& S = sub[8];
            e.cur_stream = 9;
            Ten Ud, Ld;
            alpha_halves(e, net, S, *fd, Ud, Ld);
            prD = e.projector(net, S, Ud, Ld, "xAOBy", "xB");
        }
        e.cur_stream = 0;
        e.parallel(P, std::move(sub));
    }
    const Engine::PPair &Pa = pr1[0], &Qa = pr1[1];   // [xl, B_v | k], [xr, A_v | k]
    const Engine::PPair &Pk = pr1[2], &Qk = pr1[3];   // [xl, s, B.u | k], [xr, A.d, s | k]
    const Engine::PPair &Pi = pr1[4], &Qi = pr1[5];   // [xl, s', B.u | k], [xr, A.d, s' | k]

    // stage 2: the two-column patches of the three cuts (stage-1 projectors applied), each
    // followed by its SVD pipeline, one stream per cut
    Engine::PPair pr2[3];
    {
        std::vector<Plan> sub(3);
        // alpha (2 x 2 cells): (k1, A_v, O_v | O_v', B_v', kR)
        // half (2 x 1 cells): (k1, A.d, O.d | k2, A.r, O.r) above the cut and
        // (k1, A.u, O.u | k2, B.r, O.r) below, the column-cut bra lines renormalised by the up
        // move's P_T and the down move's P_B (the lower corner's in the down move's frame: its ket
        // line); in the D2 scheme those are this move's own pair, by symmetry
        {
            Plan& S = sub[0];
            e.cur_stream = 1;
            auto D = [&](const char* spec, const Ten& X1, const Ten& Y1) { return e.ctr(net, S, spec, X1, Y1); };
            const Ten Q1 = D("hErfRZgS,kZg->hkEfrRS", Q1pre, Pa.PT);
            const Ten Q4 = D("hbSoRxpr,xbk->hkporRS", Q4pre, Pa.PB);
            if (half4) {
                const Ten U2a = D("hkEfrRS,jhS->kEfjrR", Q1, sym ? Pa.PT : prU.PT);
                const Ten L2a = D("hkporRS,hrj->kpojSR", Q4, sym ? Pa.PB : prD.PB);
                pr2[0] = e.projector(net, S, U2a, L2a, "abcdef", "abc");
            } else {
                const Ten Q2 = D("hElWfLMg,kWE->hlLMfgk", Q2pre, Qa.PT);
                const Ten U2a = D("hkEfrRS,hrRSFGK->kEfFGK", Q1, Q2);
                const Ten Q3 = D("hbMoLypl,ypk->hlLMobk", Q3pre, Qa.PB);
                const Ten L2a = D("hkporRS,hrRSOBK->kpoOBK", Q4, Q3);
                pr2[0] = e.projector(net, S, U2a, L2a, "abcdef", "abc");
            }
        }
        // kappa (1 x 2 cells): (k2, A.d, O.u | O.u', B.u', kR)
        {
            Plan& S = sub[1];
            e.cur_stream = 2;
            auto D = [&](const char* spec, const Ten& X1, const Ten& Y1) { return e.ctr(net, S, spec, X1, Y1); };
            const Ten ULk = D("hobxsEr,kxsb->hkEor", ULA, Pk.PT);
            const Ten URk = D("hobysEl,kyEs->hlobk", URA, Qk.PT);
            const Ten U2k = D("hkEor,hrOBK->kEoOBK", ULk, URk);
            const Ten LLk = D("hEbQxsoR,xsbk->hkEoRQ", LLkpre, Pk.PB);
            const Ten LRk = D("hEbMysoL,yEsk->hLMobk", LRkpre, Qk.PB);
            const Ten L2k = D("hkEoRQ,hRQOBK->kEoOBK", LLk, LRk);
            pr2[1] = e.projector(net, S, U2k, L2k, "abcdef", "abc");
        }
        // iota (1 x 2 cells): (k3, A.d, O.d | O.d', B.u', kR)
        {
            Plan& S = sub[2];
            e.cur_stream = 3;
            auto D = [&](const char* spec, const Ten& X1, const Ten& Y1) { return e.ctr(net, S, spec, X1, Y1); };
            const Ten ULi = D("hbErXtfR,kXtb->hkEfrR", ULAO, Pi.PT);
            const Ten URi = D("hbElYtfL,kYEt->hlLfbk", URAO, Qi.PT);
            const Ten U2i = D("hkEfrR,hrRFBK->kEfFBK", ULi, URi);
            const Ten LLi = D("hEfxtbQ,xtbk->hkEfQ", LLipre, Pi.PB);
            const Ten LRi = D("hEfytbM,yEtk->hMfbk", LRipre, Qi.PB);
            const Ten L2i = D("hkEfQ,hQFBK->kEfFBK", LLi, LRi);
            pr2[2] = e.projector(net, S, U2i, L2i, "abcdef", "abc");
        }
        e.cur_stream = 0;
        e.parallel(P, std::move(sub));
    }
    const Engine::PPair &P4 = pr2[0], &P5 = pr2[1], &P6 = pr2[2];

    // composite projector of each cut (stage 1 then stage 2)
    const Ten PaB = C("xbK,Kaok->xaobk", Pa.PB, P4.PB);      // [xl, A_v, O_v, B_v, k]
    const Ten PaT = C("kKao,Kxb->kxaob", P4.PT, Pa.PT);
    const Ten PkB = C("xsbK,Keok->xesobk", Pk.PB, P5.PB);    // [xl, A.d, s, O.u, B.u, k]
    const Ten PkT = C("kKeo,Kxsb->kxesob", P5.PT, Pk.PT);
    const Ten PiB = C("xtbK,Kefk->xeftbk", Pi.PB, P6.PB);    // [xl, A.d, O.d, s', B.u, k]
    const Ten PiT = C("kKef,Kxtb->kxeftb", P6.PT, Pi.PT);

    // renormalisation (Fig. 5(c)); crossing lines are summed between the two projectors
    Ten C1n, C4n;
    if (sym) {
        // Q1pre is C1 with one column (T1^{k,i,b}) and one row (T4^{k,i,b} and the site)
        // absorbed, [h, A.d, A.r, O.d, O.r, v, B.d, B.r]; P_T truncates its row-cut group
        // (v, A.d, O.d, B.d) and, read in the diagonally reflected frame, its column-cut group
        // (h, A.r, O.r, B.r).  Q4pre, [h, B.u, B.r, O.u, O.r, v, A.u, A.r], is the same for C4
        // (bottom edge, last row); P_B truncates (v, A.u, O.u, B.u) and, in the frame reflected
        // about the anti-diagonal (which exchanges ket and bra), (h, B.r, O.r, A.r).
        X = C("hErfRZgS,kZEfg->hrRSk", Q1pre, PaT);
        C1n = C("hrRSk,jhrRS->jk", X, PaT);
        X = C("hbSoRxpr,xpobk->hSRrk", Q4pre, PaB);
        C4n = C("hSRrk,hSRrj->jk", X, PaB);
        double *c1 = C1n.p, *c4 = C4n.p;
        const int n = net.chi;
        e.push(P, std::make_unique<FnStep>([=](cudaStream_t s) {
            launch_symmetrize(c1, n, s);
            launch_symmetrize(c4, n, s);
        }));
    } else {
        C1n = C("hvpob,kvpob->hk", Ct1, PaT);
        C4n = C("hvEfg,vEfgk->hk", Ct4, PaB);
    }
    X = C("xpobK,xXl->pobKXl", PaB, T4k);
    X = C("pobKXl,splEr->obKXsEr", X, A);
    const Ten T4kn = C("obKXsEr,kXEsob->Kkr", X, PkT);
    X = C("xEsobK,xXL->EsobKXL", PkB, T4i);
    X = C("EsobKXL,tsoLfR->EbKXtfR", X, O);
    const Ten T4in = C("EbKXtfR,kXEftb->KkR", X, PiT);
    X = C("xEftbK,xXM->EftbKXM", PiB, T4b);
    X = C("EftbKXM,tbMgS->EfKXgS", X, B);
    const Ten T4bn = C("EfKXgS,kXEfg->KkS", X, PaT);

    // Frobenius normalisation, written back through the frame's views of C1, T4, C4
    std::vector<NormItem> items;
    auto item = [](const Ten& src, const Ten& dst) {
        NormItem it;
        it.src = src.p;
        it.dst = dst.p;
        it.d0 = src.dim[0];
        it.d1 = src.nd > 1 ? src.dim[1] : 1;
        it.d2 = src.nd > 2 ? src.dim[2] : 1;
        it.s0 = dst.st[0];
        it.s1 = dst.nd > 1 ? dst.st[1] : 0;
        it.s2 = dst.nd > 2 ? dst.st[2] : 0;
        return it;
    };
    items.push_back(item(C1n, f.C[0]));
    items.push_back(item(T4kn, f.T[3][0]));
    items.push_back(item(T4in, f.T[3][1]));
    items.push_back(item(T4bn, f.T[3][2]));
    items.push_back(item(C4n, f.C[3]));
    NormItem* dev = (NormItem*)e.dalloc((long long)(items.size() * sizeof(NormItem) + 7) / 8);
    if (!e.dry)
        CUDA_OK(cudaMemcpy(dev, items.data(), items.size() * sizeof(NormItem),
                           cudaMemcpyHostToDevice));
    const int cnt = (int)items.size();
    e.push(P, std::make_unique<FnStep>([=](cudaStream_t s) { launch_normalize(dev, cnt, s); }));
    if (e.tape) {
        TapeOp op;
        op.kind = TapeOp::NORM;
        op.items = {{C1n, f.C[0]}, {T4kn, f.T[3][0]}, {T4in, f.T[3][1]}, {T4bn, f.T[3][2]},
                    {C4n, f.C[3]}};
        e.tape->push_back(op);
    }
}

// convergence check (Sec. III.D): singular values of rho_eff = C1 C2 C3 C4 / Tr
void build_spectrum(Engine& e, Network& net) {
    Plan& P = net.spectrum;
    const int chi = net.chi;
    const Ten R1 = e.ctr(net, P, "ab,ac->bc", net.C[0], net.C[1]);
    const Ten R2 = e.ctr(net, P, "bc,dc->bd", R1, net.C[2]);
    const Ten rho = e.ctr(net, P, "bd,de->be", R2, net.C[3]);
    double* Sraw = e.dalloc(chi);
    double* rho_p = rho.p;
    double* S_old = net.S_old;
    double* dS = net.dS;
    if (e.svd_mode == SCTM_SVD_PARTIAL_RANDOM && chi <= kPsvdMaxK) {
        // singular values by the partial SVD's Jacobi kernel (the same values for rho and its
        // transpose), so that this mode makes no cuSOLVER call at all
        double* Ub = e.dalloc((long long)chi * chi);
        double* Wb = e.dalloc((long long)chi * chi);
        const int kp = chi + (chi & 1);
        double* Vg = chi > kPsvdSmemK ? e.dalloc((long long)kp * (kp + 1)) : nullptr;
        const int info_idx = net.n_svd++;
        const Network* np = &net;
        const bool jc = e.jacobi_cluster;
        e.push(P, std::make_unique<FnStep>([=](cudaStream_t s) {
            launch_jacobi_svd(rho_p, chi, Sraw, Ub, Wb, np->svd_info + info_idx, Vg, jc, s);
        }, SCTM_KERNEL_JACOBI));
        e.push(P, std::make_unique<FnStep>(
            [=](cudaStream_t s) { launch_spectrum_update(Sraw, rho_p, chi, S_old, dS, s); }));
        return;
    }
    double* work = e.dalloc((long long)chi * chi);
    e.push(P, std::make_unique<FnStep>(
        [=](cudaStream_t s) { launch_copy(rho_p, work, (long long)chi * chi, s); }));
    auto sv = std::make_unique<SvdStep>();
    sv->M = work;
    sv->n = chi;
    sv->S = Sraw;
    sv->U = work;
    sv->V = work;
    sv->vectors = false;
    sv->net = &net;
    sv->info_idx = net.n_svd++;
    net.svd_nmax = std::max(net.svd_nmax, chi);
    net.svd_steps.push_back(sv.get());
    e.push(P, std::move(sv));
    e.push(P, std::make_unique<FnStep>(
        [=](cudaStream_t s) { launch_spectrum_update(Sraw, rho_p, chi, S_old, dS, s); }));
}

// Z00, Z10, Z01, Z11, ln kappa and the bra environment E (Sec. II, Fig. 4(b),(c))
static void build_local(Engine& e, Network& net) {
    Plan& P = net.local;
    auto C = [&](const char* spec, const Ten& X, const Ten& Y, const Ten* out = nullptr) {
        return e.ctr(net, P, spec, X, Y, out);
    };
    const Ten &C1 = net.C[0], &C2 = net.C[1], &C3 = net.C[2], &C4 = net.C[3];
    const Ten &T1k = net.T[0][0], &T1i = net.T[0][1], &T1b = net.T[0][2];
    const Ten &T2k = net.T[1][0], &T2i = net.T[1][1], &T2b = net.T[1][2];
    const Ten &T3k = net.T[2][0], &T3i = net.T[2][1], &T3b = net.T[2][2];
    const Ten &T4k = net.T[3][0], &T4i = net.T[3][1], &T4b = net.T[3][2];
    Ten X;
    X = C("av,abx->vbx", C1, T1k);
    X = C("vbx,bcy->vcxy", X, T1i);
    X = C("vcxy,cez->vexyz", X, T1b);
    const Ten Ctop = C("vexyz,ew->vxyzw", X, C2);
    X = C("av,abx->vbx", C4, T3k);
    X = C("vbx,bcy->vcxy", X, T3i);
    X = C("vcxy,cez->vexyz", X, T3b);
    const Ten Cbot = C("vexyz,ew->vxyzw", X, C3);
    const Ten Z10 = C("vxyzw,vxyzw->", Ctop, Cbot);
    const Ten X1 = C("hv,hw->vw", C1, C2);
    const Ten X2 = C("hv,hw->vw", C4, C3);
    const Ten Z00 = C("vw,vw->", X1, X2);
    X = C("hv,vbx->hbx", C1, T4k);
    X = C("hbx,bcy->hcxy", X, T4i);
    X = C("hcxy,cez->hexyz", X, T4b);
    const Ten Lrow = C("hexyz,ge->hxyzg", X, C4);
    X = C("hv,vbx->hbx", C2, T2k);
    X = C("hbx,bcy->hcxy", X, T2i);
    X = C("hcxy,cez->hexyz", X, T2b);
    const Ten Rrow = C("hexyz,ge->hxyzg", X, C3);
    const Ten Z01 = C("hxyzg,hxyzg->", Lrow, Rrow);
    X = C("vaobw,vxl->xaoblw", Ctop, T4k);
    X = C("xaoblw,saler->xobwser", X, net.A);
    const Ten Uk = C("xobwser,wyr->xesoby", X, T2k);
    X = C("xesoby,xXl->Xesobyl", Uk, T4i);
    X = C("Xesobyl,tsolfr->Xebyftr", X, net.O);
    const Ten Ui = C("Xebyftr,yYr->XeftbY", X, T2i);
    X = C("vefgw,xvl->xefgwl", Cbot, T4b);
    X = C("xefgwl,tblgr->xefwtbr", X, net.B);
    const Ten Li = C("xefwtbr,ywr->xeftby", X, T2b);
    X = C("XeftbY,xXl->xeftbYl", Li, T4i);
    X = C("xeftbYl,tsolfr->xebYsor", X, net.O);
    const Ten Lk = C("xebYsor,yYr->xesoby", X, T2i);
    const Ten Z11 = C("xesoby,xesoby->", Uk, Lk);
    X = C("xeftby,xvl->eftbylv", Ui, T4b);
    X = C("eftbylv,vefgw->tbylgw", X, Cbot);
    C("tbylgw,ywr->tblgr", X, T2b, &net.E);
    double *z00 = Z00.p, *z10 = Z10.p, *z01 = Z01.p, *z11 = Z11.p, *lnk = net.lnk;
    net.z[0] = z00;
    net.z[1] = z10;
    net.z[2] = z01;
    net.z[3] = z11;
    e.push(P, std::make_unique<FnStep>(
        [=](cudaStream_t s) { launch_lnkappa(z00, z10, z01, z11, lnk, s); }));
    if (e.tape) {
        TapeOp op;
        op.kind = TapeOp::LNK;
        op.z[0] = z00;
        op.z[1] = z10;
        op.z[2] = z01;
        op.z[3] = z11;
        e.tape->push_back(op);
    }
}

bool Engine::all_warm(const Network& net) const {
    if (net.psvd_steps.empty()) return false;
    for (const PartialSvdStep* p : net.psvd_steps)
        if (!p->is_warm || !p->can_warm) return false;
    return true;
}

bool Engine::capture_iteration(Network& net) {
    if (dry || serial || profile) return false;
    cudaStream_t cs = cap_stream[cur_lane];
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    const long long before = kernel_launches.load();
    capturing = true;
    bool ok = true;
    try {
        for (int m = 0; m < 4; ++m) run(net.move[m]);
        run(net.spectrum);
    } catch (...) {
        ok = false;
    }
    capturing = false;
    cudaGraph_t g = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(cs, &g);
    // the capture only recorded launches: take them back out of the running launch count
    const long long recorded = kernel_launches.load() - before;
    kernel_launches -= recorded;
    if (!ok || ee != cudaSuccess || !g) {
        cudaGetLastError();
        if (g) cudaGraphDestroy(g);
        return false;
    }
    cudaGraphExec_t ex = nullptr;
    if (cudaGraphInstantiate(&ex, g, 0) != cudaSuccess) {
        cudaGetLastError();
        cudaGraphDestroy(g);
        return false;
    }
    if (net.graph_exec) cudaGraphExecDestroy(net.graph_exec);
    if (net.graph) cudaGraphDestroy(net.graph);
    net.graph = g;
    net.graph_exec = ex;
    net.graph_launches = recorded;
    return true;
}

void Engine::cold_svd(Network& net) {
    for (PartialSvdStep* p : net.psvd_steps) p->is_warm = false;
}

void Engine::init_env(Network& net, unsigned long long seed) {
    cold_svd(net);
    if (dry) return;
    CUDA_OK(cudaMemsetAsync(dev_err, 0, 2 * sizeof(int), stream));
    if (net.method == SCTM_METHOD_SPLIT_D2) {
        // the stored C1, C4 and T4 take the directional cold start's draws of their slots (0, 3
        // and 13..15); the corners are symmetrised, the other slots are views of these
        launch_splitmix_fill(net.C[0].p, net.C[0].numel(), seed, 0, stream);
        launch_splitmix_fill(net.C[3].p, net.C[3].numel(), seed, 3, stream);
        for (int x = 0; x < 3; ++x)
            launch_splitmix_fill(net.T[3][x].p, net.T[3][x].numel(), seed, 13 + x, stream);
        launch_symmetrize(net.C[0].p, net.chi, stream);
        launch_symmetrize(net.C[3].p, net.chi, stream);
        launch_zero(net.S_old, net.chi, stream);
        CUDA_OK(cudaGetLastError());
        return;
    }
    unsigned long long q = 0;
    for (int i = 0; i < 4; ++i) launch_splitmix_fill(net.C[i].p, net.C[i].numel(), seed, q++, stream);
    for (int i = 0; i < 4; ++i)
        for (int x = 0; x < 3; ++x)
            launch_splitmix_fill(net.T[i][x].p, net.T[i][x].numel(), seed, q++, stream);
    launch_zero(net.S_old, net.chi, stream);
    CUDA_OK(cudaGetLastError());
}

void Engine::build_network(Network& net) {
    const int chi = net.chi, D = net.D, d = net.d;
    const bool sym = net.method == SCTM_METHOD_SPLIT_D2;
    if (sym) {
        // D2-symmetric environment (Sec. III.B, Eq. "Symmetry constraints"): only C1, C4 and the
        // left edge are stored; C3 = C1, C2 = C4 (both symmetric), T1 = T4, and T2 = T3 = T4
        // with ket <-> bra and the two chain bonds exchanged, as strided views
        net.C[0] = alloc({chi, chi});
        net.C[3] = alloc({chi, chi});
        net.T[3][0] = alloc({chi, chi, D});
        net.T[3][1] = alloc({chi, chi, d});
        net.T[3][2] = alloc({chi, chi, D});
        net.C[1] = net.C[3];
        net.C[2] = net.C[0];
        for (int x = 0; x < 3; ++x) {
            net.T[0][x] = net.T[3][x];
            net.T[1][x] = permute(net.T[3][2 - x], {1, 0, 2});
            net.T[2][x] = net.T[1][x];
        }
    } else {
        for (int i = 0; i < 4; ++i) net.C[i] = alloc({chi, chi});
        for (int i = 0; i < 4; ++i) {
            net.T[i][0] = alloc({chi, chi, D});
            net.T[i][1] = alloc({chi, chi, d});
            net.T[i][2] = alloc({chi, chi, D});
        }
    }
    net.S_old = dalloc(chi);
    net.dS = dalloc(1);
    net.lnk = dalloc(2);
    net.E = alloc({net.p, D, D, D, D});
    mixed_build = true;
    if (sym) {  // one update per iteration (moves 1..3 stay empty)
        build_left_move(*this, net, net.move[SCTM_MOVE_LEFT], make_frame(net, SCTM_MOVE_LEFT), true);
    } else {
        // the up and down moves seen from each move (left, right, up, down): the frames of
        // (up, down), (down, up), (left, right), (right, left)
        const int perp_up[4] = {SCTM_MOVE_UP, SCTM_MOVE_DOWN, SCTM_MOVE_LEFT, SCTM_MOVE_RIGHT};
        const int perp_down[4] = {SCTM_MOVE_DOWN, SCTM_MOVE_UP, SCTM_MOVE_RIGHT, SCTM_MOVE_LEFT};
        for (int m = 0; m < 4; ++m) {
            tape = &net.tape_move[m];
            if (net.p4_half) {
                const Frame fu = make_frame(net, perp_up[m]), fd = make_frame(net, perp_down[m]);
                build_left_move(*this, net, net.move[m], make_frame(net, m), false, &fu, &fd);
            } else {
                build_left_move(*this, net, net.move[m], make_frame(net, m));
            }
        }
    }
    mixed_build = false;
    tape = nullptr;
    build_spectrum(*this, net);
    tape = sym ? nullptr : &net.tape_local;
    build_local(*this, net);
    tape = nullptr;
    finalize(net);
    if (precision == SCTM_PREC_F64EMU) autotune(net);
    set_precision(net, precision);
}

double Engine::cutoff_floor(int prec) {
    switch (prec) {
        // Singular values of rho_B rho_T below the form's relative error of that product are
        // noise, and S^-1/2 would amplify their vectors: measured on D=2, chi=16 (Ising,
        // T=4.6), a cutoff of 1e-6 for the hi/lo forms let such directions through and moved
        // ln kappa by 1e-2 against FP64 at the same cutoff, while 1e-3 (TF32) and 1e-2 (BF16)
        // kept the plain forms within 3e-4.
        case SCTM_PREC_TF32: return 1e-3;    // 11-bit significand
        case SCTM_PREC_BF16: return 1e-2;    // 8-bit significand
        case SCTM_PREC_TF32X3: return 1e-4;  // hi/lo, FP32 accumulation
        case SCTM_PREC_BF16X3: return 1e-3;
        default: return 0.0;  // FP64 and its emulation
    }
}

double Engine::switch_level(int prec) {
    // spectrum change below which a mixed-form iteration has reached the form's rounding level
    switch (prec) {
        case SCTM_PREC_TF32: return 1e-4;
        case SCTM_PREC_BF16: return 1e-3;
        case SCTM_PREC_TF32X3: return 1e-6;
        case SCTM_PREC_BF16X3: return 1e-5;
        default: return 0.0;
    }
}

// Which kernel runs each FP64-accurate contraction: the FP64 kernels or the FP64 emulation on
// the tensor cores.  The emulation pays off where its fixed costs (digit split of both operands,
// row exponents, one accumulator read-back per 128 K) are small against the multiply-adds it
// moves to the tensor cores, which depends on M, N, K and the batch together; so it is measured.
// autotune() times both kernels once per distinct contraction shape on this context's own buffers
// (one launch to warm up, then the best of three, CUDA events on the caller's stream) and keeps
// the faster; shapes below 4 MFLOP stay FP64 untimed (launch overheads dominate there).  The
// decisions are kept per device and shape for the life of the process, so later contexts (a
// batched sweep) reuse them.
namespace {
struct TuneChoice {
    bool emu;
    float t64, temu;
};
// decisions per (device, M, N, K, batch), shared by every context of the process
std::mutex g_tune_mutex;
std::map<std::tuple<int, int, int, int, int>, TuneChoice> g_tune;
}  // namespace

void Engine::autotune(Network& net) {
    if (dry) return;
    using Choice = TuneChoice;
    int dev = 0;
    CUDA_OK(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    std::map<std::tuple<int, int, int, int, int>, Choice>& seen = g_tune;
    cudaStream_t s = lanes[0].streams[0];
    cudaEvent_t e0, e1;
    CUDA_OK(cudaEventCreate(&e0));
    CUDA_OK(cudaEventCreate(&e1));
    auto time_it = [&](CtrLaunch a, int prec) {
        a.precision = prec;
        if (prec != SCTM_PREC_FP64) {  // the tensor-core paths split K with their own tiles
            a.splits = a.tc_splits;
            a.kchunk = a.tc_kchunk;
        }
        launch_ctr(a, s);
        float best = 1e30f;
        for (int r = 0; r < 3; ++r) {
            cudaEventRecord(e0, s);
            launch_ctr(a, s);
            cudaEventRecord(e1, s);
            CUDA_OK(cudaEventSynchronize(e1));
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            best = std::min(best, ms);
        }
        return best;
    };
    net.tuned_emu = 0;
    net.tuned_total = 0;
    for (CtrStep* st : net.ctr_steps) {
        st->emu_ok = false;
        if (!st->mixed_ok) continue;
        ++net.tuned_total;
        if (st->flops < 4000000LL) continue;
        const auto key = std::make_tuple(dev, st->a.M, st->a.N, st->a.K, st->a.nb);
        auto it = seen.find(key);
        if (it == seen.end()) {
            Choice c;
            c.t64 = time_it(st->a, SCTM_PREC_FP64);
            c.temu = time_it(st->a, SCTM_PREC_F64EMU);
            c.emu = c.temu < 0.9f * c.t64;
            it = seen.emplace(key, c).first;
            if (const char* tf = getenv("SCTM_AUTOTUNE_LOG")) {
                if (tf[0]) {
                    if (FILE* fp = fopen(tf, "a")) {
                        fprintf(fp, "%d %d %d %d %d %.4f %.4f %d\n", net.d, st->a.M, st->a.N,
                                st->a.K, st->a.nb, c.t64, c.temu, c.emu ? 1 : 0);
                        fclose(fp);
                    }
                }
            }
        }
        st->emu_ok = it->second.emu;
        if (st->emu_ok) ++net.tuned_emu;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    CUDA_OK(cudaGetLastError());
    int err[2] = {0, 0};
    CUDA_OK(cudaMemcpy(err, dev_err, sizeof(err), cudaMemcpyDeviceToHost));
    if (err[0]) throw Error(SCTM_ETIMEOUT, "autotune: a tensor-core contraction wait timed out");
}

void Engine::set_precision(Network& net, int prec) {
    for (CtrStep* s : net.ctr_steps) {
        int p = s->mixed_ok ? prec : SCTM_PREC_FP64;
        if (p == SCTM_PREC_F64EMU && !s->emu_ok) p = SCTM_PREC_FP64;
        s->a.precision = p;
    }
    net.precision = prec;
    net.cutoff_now = std::max(cutoff, cutoff_floor(prec));
}

void Engine::finalize(Network& net) {
    for (int k = 0; k < kStreams; ++k)
        if (net.splitk_need[k] > 0) net.splitk_ws[k] = dalloc((long long)net.splitk_need[k]);
    for (CtrStep* s : net.ctr_steps)
        if (s->partial_need > 0) s->a.partial = net.splitk_ws[s->sid];
    size_t px[kStreams] = {0}, py[kStreams] = {0}, pe[kStreams] = {0};
    for (CtrStep* s : net.ctr_steps) {
        if (!s->mixed_ok) continue;
        px[s->sid] = std::max({px[s->sid], tc_pack_bytes_x(s->a), emu_pack_bytes_x(s->a)});
        py[s->sid] = std::max({py[s->sid], tc_pack_bytes_y(s->a), emu_pack_bytes_y(s->a)});
        pe[s->sid] = std::max(pe[s->sid], emu_exp_ints(s->a));
    }
    for (int k = 0; k < kStreams; ++k) {
        if (px[k] > 0) net.pack_x[k] = dalloc((long long)((px[k] + 7) / 8));
        if (py[k] > 0) net.pack_y[k] = dalloc((long long)((py[k] + 7) / 8));
        if (pe[k] > 0) net.rexp[k] = (int*)dalloc((long long)((pe[k] + 1) / 2));
    }
    for (CtrStep* s : net.ctr_steps) {
        if (!s->mixed_ok) continue;
        if (!net.scale_ws[s->sid]) net.scale_ws[s->sid] = dalloc(2 * kScaleBlocks);
        s->a.scale_ws = net.scale_ws[s->sid];
        s->a.pack_x = net.pack_x[s->sid];
        s->a.pack_y = net.pack_y[s->sid];
        s->a.rexp = net.rexp[s->sid];
    }
    void* p = nullptr;
    if (!dry) {
        CUDA_OK(cudaMalloc(&p, std::max(net.n_svd, 1) * sizeof(int)));
        allocs_.push_back(p);
        CUDA_OK(cudaMemset(p, 0, std::max(net.n_svd, 1) * sizeof(int)));
    }
    net.svd_info = (int*)p;
    if (dry) return;
    const int n = net.svd_nmax;
    double* A = dalloc((long long)n * n);
    double* S = dalloc(n);
    size_t dbytes = 0, hbytes = 0;
    SOLVER_OK(cusolverDnXgesvdp_bufferSize(lanes[0].solver[0], solver_params, CUSOLVER_EIG_MODE_VECTOR, 1, n,
                                           n, CUDA_R_64F, A, n, CUDA_R_64F, S, CUDA_R_64F, A, n,
                                           CUDA_R_64F, A, n, CUDA_R_64F, &dbytes, &hbytes));
    int lwork = 0;
    SOLVER_OK(cusolverDnDgesvd_bufferSize(lanes[0].solver[0], n, n, &lwork));
    net.svd_lwork = std::max(lwork, 1);
    net.svd_dbytes = std::max<size_t>(std::max<size_t>(dbytes, 8), (size_t)net.svd_lwork * 8);
    net.svd_hbytes = std::max<size_t>(hbytes, 8);
    for (int k = 0; k < kStreams; ++k) {
        net.svd_dwork[k] = dalloc((long long)(net.svd_dbytes + 7) / 8);
        net.svd_rwork[k] = dalloc(n);
        net.svd_hwork[k].assign(net.svd_hbytes, 0);
    }
}

}  // namespace sctm
