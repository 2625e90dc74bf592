// The C ABI of libsctm.so (declared in include/sctm.h).
#include <cmath>
#include <cstring>
#include <memory>
#include <string>
#include <thread>
#include <vector>

#include "engine.h"

using namespace sctm;

struct sctm_ctx {
    std::unique_ptr<Engine> eng;
    Network net[2];
    sctm_opts opts{};
    int chi = 0;
    double* A_dev = nullptr;
    double* A_stage = nullptr;
    double* O_dev = nullptr;
    double* Oid_dev = nullptr;
    double* f_dev = nullptr;
    double* g_dev = nullptr;
    int* flag_dev = nullptr;
    cudaEvent_t lane_fork = nullptr, lane_join = nullptr;
    std::string err;
    ~sctm_ctx() {
        if (lane_fork) cudaEventDestroy(lane_fork);
        if (lane_join) cudaEventDestroy(lane_join);
    }
    bool converged = true;
    // gradient mode (SCTM_GRAD_*) and the adjoint solve's settings and last statistics
    int grad_mode = SCTM_GRAD_ENV;
    double adj_tol = 1e-10;
    int adj_max_mv = 400;
    int adj_mv[2] = {0, 0};
    double adj_res[2] = {0.0, 0.0};
    double* adj_d[2] = {nullptr, nullptr};  // d ln kappa / dA of each network (device)
};

namespace {

const char* kNullCtx = "sctm: NULL context";

#define API_BEGIN(ctx)                  \
    if (!(ctx)) return SCTM_EINVAL;     \
    (ctx)->err.clear();                 \
    try {
#define API_END(ctx)                                             \
    }                                                            \
    catch (const Error& e) {                                     \
        (ctx)->err = e.what();                                   \
        return e.code;                                           \
    }                                                            \
    catch (const std::exception& e) {                            \
        (ctx)->err = e.what();                                   \
        return SCTM_ECUDA;                                       \
    }

void check_cuda(const char* what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) throw Error(SCTM_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

void cuda_ok(cudaError_t e, const char* what) {
    if (e != cudaSuccess)
        throw Error(e == cudaErrorMemoryAllocation ? SCTM_ENOMEM : SCTM_ECUDA,
                    std::string(what) + ": " + cudaGetErrorString(e));
}

long long peps_size(const sctm_opts& o) { return (long long)o.p * o.D * o.D * o.D * o.D; }
long long pepo_size(const sctm_opts& o) { return (long long)o.p * o.p * o.d * o.d * o.d * o.d; }

// guard on entry: a PEPS with a non-finite entry never reaches an SVD
bool peps_is_finite(sctm_ctx* c, const double* dev) {
    launch_check_finite(dev, peps_size(c->opts), c->flag_dev, c->eng->stream);
    int flag = 1;
    cuda_ok(cudaMemcpyAsync(&flag, c->flag_dev, sizeof(int), cudaMemcpyDeviceToHost, c->eng->stream),
            "finite flag copy");
    cuda_ok(cudaStreamSynchronize(c->eng->stream), "finite flag sync");
    return flag == 0;
}

void check_svd_info(sctm_ctx* c) {
    for (int n = 0; n < 2; ++n) {
        Network& net = c->net[n];
        std::vector<int> info(std::max(net.n_svd, 1));
        cuda_ok(cudaMemcpyAsync(info.data(), net.svd_info, info.size() * sizeof(int),
                                cudaMemcpyDeviceToHost, c->eng->stream),
                "svd info copy");
        cuda_ok(cudaStreamSynchronize(c->eng->stream), "stream sync");
        for (int v : info)
            if (v != 0)
                throw Error(SCTM_ECUSOLVER, "gesvd reported info=" + std::to_string(v) +
                                                (n ? " (norm network)" : " (numerator network)"));
    }
}

// The two generators of the D2 symmetry that the symmetric split method relies on (Sec. III.B):
// the reflection about the main diagonal (u <-> l, d <-> r) and the 180-degree rotation (u <-> d,
// l <-> r) with the exchange s_up <-> s_dn, each to 1e-12 of max|O|.
bool pepo_has_d2_symmetry(const double* pepo, const sctm_opts& o) {
    const long long no = pepo_size(o);
    std::vector<double> h((size_t)no);
    cuda_ok(cudaMemcpy(h.data(), pepo, no * sizeof(double), cudaMemcpyDefault), "copy pepo");
    const int p = o.p, d = o.d;
    auto at = [&](int t, int s, int u, int l, int dd, int r) {
        return h[((((((size_t)t * p + s) * d + u) * d + l) * d + dd) * d + r)];
    };
    double mx = 0.0, dev = 0.0;
    for (double v : h) mx = std::max(mx, std::fabs(v));
    for (int t = 0; t < p; ++t)
        for (int s = 0; s < p; ++s)
            for (int u = 0; u < d; ++u)
                for (int l = 0; l < d; ++l)
                    for (int dd = 0; dd < d; ++dd)
                        for (int r = 0; r < d; ++r) {
                            const double v = at(t, s, u, l, dd, r);
                            dev = std::max(dev, std::fabs(v - at(t, s, l, u, r, dd)));
                            dev = std::max(dev, std::fabs(v - at(s, t, dd, r, u, l)));
                        }
    return dev <= 1e-12 * mx;
}

// cold start of one network (and, for the reduced method, the fused site tensor from A)
void init_network(sctm_ctx* c, int n) {
    Network& net = c->net[n];
    if (net.method == SCTM_METHOD_REDUCED) {
        c->eng->run(net.site);
        c->eng->init_reduced_env(net);
    } else {
        c->eng->init_env(net, c->opts.init_seed);
    }
}

}  // namespace

extern "C" {

sctm_status sctm_default_opts(sctm_opts* o) {
    if (!o) return SCTM_EINVAL;
    std::memset(o, 0, sizeof(*o));
    o->T = 1.0;
    o->D = 2;
    o->p = 2;
    o->d = 2;
    o->precision = SCTM_PREC_FP64;
    o->grad_mode = SCTM_GRAD_ENV;
    o->svd_cutoff = 1e-12;
    o->init_seed = 0;
    o->batch = 1;
    o->cuda_stream = nullptr;
    o->svd_mode = SCTM_SVD_QR;
    return SCTM_OK;
}

sctm_status sctm_ising_pepo(double T, double* O64) {
    if (!O64 || !(T > 0.0)) return SCTM_EINVAL;
    const double b = std::isinf(T) ? 0.0 : 1.0 / T;
    // sqrt(W): eigenvalues 2cosh(b) on (1,1)/sqrt2 and 2sinh(b) on (1,-1)/sqrt2 (Sec. IV)
    const double cp = std::sqrt(2.0 * std::cosh(b)), sm = std::sqrt(2.0 * std::sinh(b));
    const double Q[2][2] = {{0.5 * (cp + sm), 0.5 * (cp - sm)}, {0.5 * (cp - sm), 0.5 * (cp + sm)}};
    for (int i = 0; i < 64; ++i) {
        int idx[6];
        for (int k = 0; k < 6; ++k) idx[k] = (i >> (5 - k)) & 1;
        double v = 0.0;
        for (int s = 0; s < 2; ++s) {
            double t = 1.0;
            for (int k = 0; k < 6; ++k) t *= Q[s][idx[k]];
            v += t;
        }
        O64[i] = v;
    }
    return SCTM_OK;
}

sctm_status sctm_create(const double* peps, const double* pepo, int chi, const sctm_opts* o,
                        sctm_ctx** out) {
    if (!out) return SCTM_EINVAL;
    *out = nullptr;
    if (!peps || !pepo) return SCTM_EINVAL;
    sctm_opts opts;
    if (o) opts = *o; else sctm_default_opts(&opts);
    if (chi < 1 || chi > 4096 || opts.D < 1 || opts.p < 1 || opts.d < 1 || opts.batch != 1 ||
        opts.precision < SCTM_PREC_FP64 || opts.precision > SCTM_PREC_F64EMU ||
        (opts.grad_mode != SCTM_GRAD_ENV && opts.grad_mode != SCTM_GRAD_ADJOINT) ||
        !(opts.svd_cutoff >= 0.0) || opts.D > 64 || opts.d > 64 || opts.p > 64 ||
        opts.svd_mode < SCTM_SVD_QR || opts.svd_mode > SCTM_SVD_PARTIAL_RANDOM ||
        (opts.method != SCTM_METHOD_SPLIT && opts.method != SCTM_METHOD_REDUCED &&
         opts.method != SCTM_METHOD_SPLIT_D2) ||
        (opts.method == SCTM_METHOD_REDUCED &&
         (opts.precision != SCTM_PREC_FP64 || opts.grad_mode != SCTM_GRAD_ENV)) ||
        (opts.method == SCTM_METHOD_SPLIT_D2 && opts.grad_mode != SCTM_GRAD_ENV) ||
        (opts.p4_mode != SCTM_P4_FULL && opts.p4_mode != SCTM_P4_HALF) ||
        (opts.p4_mode == SCTM_P4_HALF &&
         (opts.method == SCTM_METHOD_REDUCED || opts.grad_mode != SCTM_GRAD_ENV)) ||
        (opts.jacobi != SCTM_JACOBI_CTA && opts.jacobi != SCTM_JACOBI_CLUSTER))
        return SCTM_EINVAL;
    std::unique_ptr<sctm_ctx> c(new sctm_ctx());
    c->opts = opts;
    c->chi = chi;
    c->grad_mode = opts.grad_mode;
    try {
        cudaStream_t s = (cudaStream_t)opts.cuda_stream;
        c->eng.reset(new Engine(s, opts.precision, opts.svd_cutoff));
        c->eng->svd_mode = opts.svd_mode;
        c->eng->jacobi_cluster = opts.jacobi == SCTM_JACOBI_CLUSTER;
        Engine& e = *c->eng;
        const long long na = peps_size(opts), no = pepo_size(opts);
        c->A_dev = e.dalloc(na);
        c->O_dev = e.dalloc(no);
        c->Oid_dev = e.dalloc((long long)opts.p * opts.p);
        c->f_dev = e.dalloc(1);
        c->g_dev = e.dalloc(na);
        c->flag_dev = (int*)e.dalloc(1);
        if (!e.dry)
            cuda_ok(cudaMemcpy(c->A_dev, peps, na * sizeof(double), cudaMemcpyDefault),
                    "copy peps");
        c->A_stage = e.dalloc(na);
        if (!e.dry) {
            if (!peps_is_finite(c.get(), c->A_dev)) return SCTM_ENUMERIC;
            if (opts.method == SCTM_METHOD_SPLIT_D2) {
                if (!pepo_has_d2_symmetry(pepo, opts)) return SCTM_EINVAL;
                launch_copy(c->A_dev, c->A_stage, na, s);
                launch_d4_project(c->A_stage, c->A_dev, opts.p, opts.D, s);
            }
            cuda_ok(cudaMemcpy(c->O_dev, pepo, no * sizeof(double), cudaMemcpyDefault),
                    "copy pepo");
            std::vector<double> oid((size_t)opts.p * opts.p, 0.0);
            for (int i = 0; i < opts.p; ++i) oid[(size_t)i * opts.p + i] = 1.0;
            cuda_ok(cudaMemcpy(c->Oid_dev, oid.data(), oid.size() * sizeof(double),
                               cudaMemcpyHostToDevice),
                    "copy identity pepo");
        }
        for (int n = 0; n < 2; ++n) {
            Network& net = c->net[n];
            net.D = opts.D;
            net.p = opts.p;
            net.d = n == 0 ? opts.d : 1;
            net.chi = chi;
            net.A = view(c->A_dev, {opts.p, opts.D, opts.D, opts.D, opts.D});
            net.B = net.A;
            net.O = n == 0 ? view(c->O_dev, {opts.p, opts.p, opts.d, opts.d, opts.d, opts.d})
                           : view(c->Oid_dev, {opts.p, opts.p, 1, 1, 1, 1});
            net.method = opts.method;
            net.p4_half = opts.p4_mode == SCTM_P4_HALF;
            if (opts.method == SCTM_METHOD_REDUCED)
                e.build_reduced_network(net);
            else
                e.build_network(net);
        }
        if (e.dry) {  // plans only: report success without a usable context
            const char* da = getenv("SCTM_DRYRUN_ADJOINT");
            if (da && da[0] == '1' && opts.method == SCTM_METHOD_SPLIT)
                for (int n = 0; n < 2; ++n) e.build_adjoint(c->net[n]);
            c.reset();
            return SCTM_OK;
        }
        cuda_ok(cudaEventCreateWithFlags(&c->lane_fork, cudaEventDisableTiming), "event");
        cuda_ok(cudaEventCreateWithFlags(&c->lane_join, cudaEventDisableTiming), "event");
        cuda_ok(cudaDeviceSynchronize(), "plan build");
        for (int n = 0; n < 2; ++n) init_network(c.get(), n);
        cuda_ok(cudaStreamSynchronize(s), "cold start");
        check_cuda("create");
    } catch (const Error& e) {
        return e.code;
    } catch (const std::exception&) {
        return SCTM_ECUDA;
    }
    *out = c.release();
    return SCTM_OK;
}

sctm_status sctm_set_peps(sctm_ctx* ctx, const double* peps, int reset_env) {
    API_BEGIN(ctx)
    if (!peps) throw Error(SCTM_EINVAL, "NULL peps");
    const long long na = peps_size(ctx->opts);
    cuda_ok(cudaMemcpyAsync(ctx->A_stage, peps, na * sizeof(double), cudaMemcpyDefault,
                            ctx->eng->stream),
            "copy peps");
    if (!peps_is_finite(ctx, ctx->A_stage)) {
        ctx->err = "PEPS tensor has a non-finite entry (previous PEPS kept)";
        return SCTM_ENUMERIC;
    }
    if (ctx->opts.method == SCTM_METHOD_SPLIT_D2)  // kept in the D4-invariant subspace
        launch_d4_project(ctx->A_stage, ctx->A_dev, ctx->opts.p, ctx->opts.D, ctx->eng->stream);
    else
        launch_copy(ctx->A_stage, ctx->A_dev, na, ctx->eng->stream);
    for (int n = 0; n < 2; ++n) {
        if (reset_env)
            init_network(ctx, n);
        else if (ctx->net[n].method == SCTM_METHOD_REDUCED)
            ctx->eng->run(ctx->net[n].site);  // the fused site tensor follows A
    }
    check_cuda("set_peps");
    return SCTM_OK;
    API_END(ctx)
}

sctm_status sctm_iterate(sctm_ctx* ctx, int max_it, double tol, int* it_done, double* last_dS) {
    API_BEGIN(ctx)
    if (max_it < 0) throw Error(SCTM_EINVAL, "max_it < 0");
    Engine& e = *ctx->eng;
    // The two networks are independent: the norm network runs on lane 1 from a second host
    // thread, ordered after everything already on the caller's stream and joined back into it.
    int its[2] = {0, 0};
    double dss[2] = {0.0, 0.0};
    std::exception_ptr errs[2];
    auto drive = [&](int n) {
        try {
            Engine::cur_lane = e.serial ? 0 : n;
            Network& net = ctx->net[n];
            cudaStream_t s0 = e.lane().streams[0];
            double dS = INFINITY;
            int it = 0;
            // Mixed forms: iterate in the tensor-core form while the spectrum change still
            // falls, then polish in FP64; convergence is only declared on FP64 iterations.
            const int form = ctx->opts.precision;
            e.set_precision(net, form);
            // graphs bake in every launch: only for the fixed FP64-accurate forms, and only in the
            // SVD mode whose warm iteration makes no cuSOLVER call (SCTM_NO_GRAPH=1 disables them)
            const char* ng = getenv("SCTM_NO_GRAPH");
            bool use_graph = ctx->opts.svd_mode == SCTM_SVD_PARTIAL_RANDOM &&
                             (form == SCTM_PREC_FP64 || form == SCTM_PREC_F64EMU) &&
                             !(ng && ng[0] == '1');
            double best = INFINITY;
            int stall = 0;
            for (it = 1; it <= max_it; ++it) {
                // warm iterations of a capturable plan replay one captured CUDA graph
                bool replay = false;
                if (use_graph && !e.profile && !e.serial && e.all_warm(net)) {
                    if (!net.graph_exec && !e.capture_iteration(net)) use_graph = false;
                    replay = net.graph_exec != nullptr && use_graph;
                }
                if (replay) {
                    cuda_ok(cudaGraphLaunch(net.graph_exec, s0), "graph launch");
                    e.kernel_launches += net.graph_launches;
                } else {
                    for (int m = 0; m < 4; ++m) e.run(net.move[m]);
                    e.run(net.spectrum);
                }
                check_cuda("iteration");
                int err[2] = {0, 0};
                cuda_ok(cudaMemcpyAsync(&dS, net.dS, sizeof(double), cudaMemcpyDeviceToHost, s0),
                        "dS copy");
                cuda_ok(cudaMemcpyAsync(err, e.dev_err, 2 * sizeof(int), cudaMemcpyDeviceToHost, s0),
                        "error flag copy");
                cuda_ok(cudaStreamSynchronize(s0), "iteration sync");
                if (err[0]) throw Error(SCTM_ETIMEOUT, "tensor-core contraction wait timed out");
                if (err[1]) throw Error(SCTM_ENUMERIC, "non-finite projector matrix");
                if (!std::isfinite(dS)) throw Error(SCTM_ENUMERIC, "non-finite spectrum change");
                if (net.precision != SCTM_PREC_FP64 && net.precision != SCTM_PREC_F64EMU) {
                    if (dS < 0.5 * best) {
                        best = dS;
                        stall = 0;
                    } else {
                        ++stall;
                    }
                    if (dS < Engine::switch_level(form) || stall >= 3)
                        e.set_precision(net, SCTM_PREC_FP64);
                    continue;
                }
                if (tol > 0.0 && dS < tol) break;
            }
            its[n] = std::min(it, max_it);
            // a spectrum change measured on a mixed-form iteration never counts as converged
            const bool fp64_like = net.precision == SCTM_PREC_FP64 || net.precision == SCTM_PREC_F64EMU;
            dss[n] = fp64_like ? dS : std::max(dS, tol > 0.0 ? 2.0 * tol : dS);
        } catch (...) {
            errs[n] = std::current_exception();
        }
        Engine::cur_lane = 0;
    };
    // each call reports its own device-side failures (timeout, non-finite projector matrix)
    cuda_ok(cudaMemsetAsync(e.dev_err, 0, 2 * sizeof(int), e.stream), "error flags");
    if (e.serial) {  // serialised profiling: both networks on the caller's stream, in turn
        drive(0);
        drive(1);
    } else {
        cuda_ok(cudaEventRecord(ctx->lane_fork, e.stream), "fork");
        cuda_ok(cudaStreamWaitEvent(e.lanes[1].streams[0], ctx->lane_fork, 0), "fork wait");
        std::thread t1(drive, 1);
        drive(0);
        t1.join();
        cuda_ok(cudaEventRecord(ctx->lane_join, e.lanes[1].streams[0]), "join");
        cuda_ok(cudaStreamWaitEvent(e.stream, ctx->lane_join, 0), "join wait");
    }
    for (auto& x : errs)
        if (x) std::rethrow_exception(x);
    if (e.profile) e.harvest();
    check_svd_info(ctx);
    bool conv = true;
    double dS_max = 0.0;
    for (int n = 0; n < 2; ++n) {
        if (tol > 0.0 && !(dss[n] < tol)) conv = false;
        if (std::isfinite(dss[n])) dS_max = std::max(dS_max, dss[n]);
    }
    ctx->converged = conv;
    if (it_done) *it_done = std::max(its[0], its[1]);
    if (last_dS) *last_dS = dS_max;
    if (!conv) {
        ctx->err = "iteration limit reached before convergence";
        return SCTM_ENOCONV;
    }
    return SCTM_OK;
    API_END(ctx)
}

static sctm_status finish_local(sctm_ctx* ctx) {
    Engine& e = *ctx->eng;
    for (int n = 0; n < 2; ++n) e.run(ctx->net[n].local);
    check_cuda("local contractions");
    return SCTM_OK;
}

sctm_status sctm_free_energy(sctm_ctx* ctx, double* f) {
    API_BEGIN(ctx)
    if (!f) throw Error(SCTM_EINVAL, "NULL f");
    Engine& e = *ctx->eng;
    finish_local(ctx);
    launch_free_energy(ctx->net[0].lnk, ctx->net[1].lnk, ctx->opts.T, ctx->f_dev, e.stream);
    check_cuda("free energy");
    cuda_ok(cudaMemcpyAsync(f, ctx->f_dev, sizeof(double), cudaMemcpyDeviceToHost, e.stream),
            "f copy");
    cuda_ok(cudaStreamSynchronize(e.stream), "f sync");
    if (!std::isfinite(*f)) {
        ctx->err = "kappa <= 0 or not finite";
        return SCTM_ENUMERIC;
    }
    if (!ctx->converged) {
        ctx->err = "environment not converged";
        return SCTM_ENOCONV;
    }
    return SCTM_OK;
    API_END(ctx)
}

sctm_status sctm_grad(sctm_ctx* ctx, double* g) {
    API_BEGIN(ctx)
    if (!g) throw Error(SCTM_EINVAL, "NULL g");
    Engine& e = *ctx->eng;
    const int n = (int)peps_size(ctx->opts);
    if (ctx->grad_mode == SCTM_GRAD_ADJOINT) {
        // d f / d A by implicit differentiation of each network's fixed point; the recompute
        // iteration runs in FP64 (or its emulation) whatever the context's form
        cuda_ok(cudaStreamSynchronize(e.stream), "adjoint start");
        for (int k = 0; k < 2; ++k) {
            Network& net = ctx->net[k];
            if (!ctx->adj_d[k]) ctx->adj_d[k] = e.dalloc(n);
            const int prec = net.precision;
            if (prec != SCTM_PREC_FP64 && prec != SCTM_PREC_F64EMU)
                e.set_precision(net, SCTM_PREC_FP64);
            e.adjoint_lnk_grad(net, ctx->adj_d[k], ctx->adj_tol, ctx->adj_max_mv, &ctx->adj_mv[k],
                               &ctx->adj_res[k]);
        }
        finish_local(ctx);
        launch_adj_combine(ctx->adj_d[0], ctx->adj_d[1], ctx->opts.T, n, ctx->g_dev, e.stream);
    } else {
        finish_local(ctx);
        launch_grad_combine(ctx->net[0].E.p, ctx->net[0].lnk, ctx->net[1].E.p, ctx->net[1].lnk,
                            ctx->opts.T, n, ctx->g_dev, e.stream);
        if (ctx->opts.method == SCTM_METHOD_SPLIT_D2) {  // the D4 group average of g
            launch_copy(ctx->g_dev, ctx->A_stage, n, e.stream);
            launch_d4_project(ctx->A_stage, ctx->g_dev, ctx->opts.p, ctx->opts.D, e.stream);
        }
    }
    check_cuda("gradient");
    cuda_ok(cudaMemcpyAsync(g, ctx->g_dev, n * sizeof(double), cudaMemcpyDefault, e.stream),
            "g copy");
    cuda_ok(cudaStreamSynchronize(e.stream), "g sync");
    double lnk[2][2];
    for (int k = 0; k < 2; ++k)
        cuda_ok(cudaMemcpy(lnk[k], ctx->net[k].lnk, 2 * sizeof(double), cudaMemcpyDeviceToHost),
                "lnk copy");
    if (!std::isfinite(lnk[0][0]) || !std::isfinite(lnk[1][0])) {
        ctx->err = "kappa <= 0 or not finite";
        return SCTM_ENUMERIC;
    }
    if (ctx->grad_mode == SCTM_GRAD_ADJOINT &&
        !(ctx->adj_res[0] <= ctx->adj_tol && ctx->adj_res[1] <= ctx->adj_tol)) {
        ctx->err = "adjoint linear solve stopped above its tolerance";
        return SCTM_ENOCONV;
    }
    if (!ctx->converged) {
        ctx->err = "environment not converged";
        return SCTM_ENOCONV;
    }
    return SCTM_OK;
    API_END(ctx)
}

sctm_status sctm_set_grad_mode(sctm_ctx* ctx, int mode, double tol, int max_matvecs,
                               double svd_grad_cutoff) {
    API_BEGIN(ctx)
    if (mode != SCTM_GRAD_ENV && mode != SCTM_GRAD_ADJOINT) throw Error(SCTM_EINVAL, "bad mode");
    if (mode == SCTM_GRAD_ADJOINT && !(svd_grad_cutoff >= 0.0 && svd_grad_cutoff < 1.0))
        throw Error(SCTM_EINVAL, "svd_grad_cutoff must lie in [0, 1)");
    if (mode == SCTM_GRAD_ADJOINT && ctx->opts.method != SCTM_METHOD_SPLIT)
        throw Error(SCTM_EINVAL, "the adjoint gradient is built for the split method only");
    if (mode == SCTM_GRAD_ADJOINT && ctx->opts.p4_mode == SCTM_P4_HALF)
        throw Error(SCTM_EINVAL, "the adjoint gradient is built for the full projector 4 only");
    if (mode == SCTM_GRAD_ADJOINT && !(tol > 0.0 && tol < 1.0 && max_matvecs >= 1))
        throw Error(SCTM_EINVAL, "adjoint tolerance must lie in (0, 1), max_matvecs >= 1");
    ctx->grad_mode = mode;
    if (mode == SCTM_GRAD_ADJOINT) {
        ctx->adj_tol = tol;
        ctx->adj_max_mv = max_matvecs;
        for (int n = 0; n < 2; ++n) ctx->net[n].adj_gcut = svd_grad_cutoff;
    }
    return SCTM_OK;
    API_END(ctx)
}

sctm_status sctm_adjoint_info(sctm_ctx* ctx, int* matvecs, double* residual) {
    API_BEGIN(ctx)
    if (matvecs) {
        matvecs[0] = ctx->adj_mv[0];
        matvecs[1] = ctx->adj_mv[1];
    }
    if (residual) {
        residual[0] = ctx->adj_res[0];
        residual[1] = ctx->adj_res[1];
    }
    return SCTM_OK;
    API_END(ctx)
}

sctm_status sctm_destroy(sctm_ctx* ctx) {
    if (!ctx) return SCTM_OK;
    if (ctx->eng) cudaStreamSynchronize(ctx->eng->stream);
    delete ctx;
    return SCTM_OK;
}

const char* sctm_last_error(const sctm_ctx* ctx) {
    if (!ctx) return kNullCtx;
    return ctx->err.c_str();
}

size_t sctm_env_size(const sctm_ctx* ctx, int network) {
    if (!ctx || network < 0 || network > 1) return 0;
    const Network& n = ctx->net[network];
    size_t s = 0;
    for (int i = 0; i < 4; ++i) s += (size_t)n.C[i].numel();
    for (int i = 0; i < 4; ++i)
        for (int x = 0; x < 3; ++x) s += (size_t)n.T[i][x].numel();
    return s;
}

static sctm_status env_copy(sctm_ctx* ctx, int network, double* host, size_t n, bool to_host) {
    API_BEGIN(ctx)
    if (network < 0 || network > 1 || !host || n < sctm_env_size(ctx, network))
        throw Error(SCTM_EINVAL, "bad network, buffer or size");
    Network& net = ctx->net[network];
    std::vector<Ten*> ts;
    for (int i = 0; i < 4; ++i) ts.push_back(&net.C[i]);
    for (int i = 0; i < 4; ++i)
        for (int x = 0; x < 3; ++x) ts.push_back(&net.T[i][x]);
    const bool sym = net.method == SCTM_METHOD_SPLIT_D2;
    size_t off = 0;
    cuda_ok(cudaStreamSynchronize(ctx->eng->stream), "sync");
    for (size_t k = 0; k < ts.size(); ++k) {
        Ten* t = ts[k];
        const size_t cnt = (size_t)t->numel(), bytes = cnt * sizeof(double);
        // the symmetric method stores C1 (slot 0), C4 (slot 3) and T4 (slots 13..15); the other
        // slots are views of them (possibly with permuted strides)
        const bool stored = !sym || k == 0 || k == 3 || k >= 13;
        if (to_host) {
            bool contiguous = true;
            for (int i = t->nd - 1, st = 1; i >= 0; st *= t->dim[i], --i)
                contiguous = contiguous && t->st[i] == st;
            if (contiguous) {
                cuda_ok(cudaMemcpy(host + off, t->p, bytes, cudaMemcpyDeviceToHost), "env export");
            } else {  // a permuted view of a stored tensor of the same size: gather on the host
                std::vector<double> raw(cnt);
                cuda_ok(cudaMemcpy(raw.data(), t->p, bytes, cudaMemcpyDeviceToHost), "env export");
                std::vector<int> ix(t->nd, 0);
                for (size_t e = 0; e < cnt; ++e) {
                    long long o = 0;
                    for (int i = 0; i < t->nd; ++i) o += ix[i] * t->st[i];
                    host[off + e] = raw[(size_t)o];
                    for (int i = t->nd - 1; i >= 0; --i) {
                        if (++ix[i] < t->dim[i]) break;
                        ix[i] = 0;
                    }
                }
            }
        } else if (stored) {
            cuda_ok(cudaMemcpy(t->p, host + off, bytes, cudaMemcpyHostToDevice), "env import");
        }
        off += cnt;
    }
    if (!to_host && sym) {
        launch_symmetrize(net.C[0].p, net.chi, ctx->eng->stream);
        launch_symmetrize(net.C[3].p, net.chi, ctx->eng->stream);
        check_cuda("env import");
    }
    if (!to_host) ctx->eng->cold_svd(net);  // the warm-start subspaces belong to the old state
    return SCTM_OK;
    API_END(ctx)
}

sctm_status sctm_env_export(sctm_ctx* ctx, int network, double* host_buf, size_t n) {
    return env_copy(ctx, network, host_buf, n, true);
}

sctm_status sctm_env_import(sctm_ctx* ctx, int network, const double* host_buf, size_t n) {
    return env_copy(ctx, network, const_cast<double*>(host_buf), n, false);
}

sctm_status sctm_move(sctm_ctx* ctx, int network, int direction) {
    API_BEGIN(ctx)
    if (network < 0 || network > 1 || direction < 0 || direction > 3)
        throw Error(SCTM_EINVAL, "bad network or direction");
    if (ctx->opts.method == SCTM_METHOD_SPLIT_D2 && direction != SCTM_MOVE_LEFT)
        throw Error(SCTM_EINVAL, "the symmetric method has one update per iteration (LEFT)");
    ctx->eng->run(ctx->net[network].move[direction]);
    check_cuda("move");
    cuda_ok(cudaStreamSynchronize(ctx->eng->stream), "move sync");
    return SCTM_OK;
    API_END(ctx)
}

sctm_status sctm_spectrum(sctm_ctx* ctx, int network, double* S) {
    API_BEGIN(ctx)
    if (network < 0 || network > 1 || !S) throw Error(SCTM_EINVAL, "bad network or buffer");
    Network& net = ctx->net[network];
    ctx->eng->run(net.spectrum);
    check_cuda("spectrum");
    cuda_ok(cudaMemcpyAsync(S, net.S_old, net.chi * sizeof(double), cudaMemcpyDeviceToHost,
                            ctx->eng->stream),
            "spectrum copy");
    cuda_ok(cudaStreamSynchronize(ctx->eng->stream), "spectrum sync");
    return SCTM_OK;
    API_END(ctx)
}

sctm_status sctm_local_values(sctm_ctx* ctx, int network, double* out5) {
    API_BEGIN(ctx)
    if (network < 0 || network > 1 || !out5) throw Error(SCTM_EINVAL, "bad network or buffer");
    Network& net = ctx->net[network];
    ctx->eng->run(net.local);
    check_cuda("local contractions");
    for (int k = 0; k < 4; ++k)
        cuda_ok(cudaMemcpyAsync(out5 + k, net.z[k], sizeof(double), cudaMemcpyDeviceToHost,
                                ctx->eng->stream),
                "Z copy");
    cuda_ok(cudaMemcpyAsync(out5 + 4, net.lnk, sizeof(double), cudaMemcpyDeviceToHost,
                            ctx->eng->stream),
            "lnk copy");
    cuda_ok(cudaStreamSynchronize(ctx->eng->stream), "Z sync");
    return SCTM_OK;
    API_END(ctx)
}

sctm_status sctm_iterate_batch(sctm_ctx* const* ctxs, int count, int max_it, double tol,
                               int* status, int* it_done, double* last_dS) {
    if (!ctxs || count < 0) return SCTM_EINVAL;
    for (int i = 0; i < count; ++i)
        if (!ctxs[i]) return SCTM_EINVAL;
    std::vector<int> st(count, SCTM_OK), it(count, 0);
    std::vector<double> ds(count, 0.0);
    std::vector<std::thread> th;
    for (int i = 0; i < count; ++i)
        th.emplace_back([&, i] { st[i] = sctm_iterate(ctxs[i], max_it, tol, &it[i], &ds[i]); });
    for (auto& t : th) t.join();
    sctm_status worst = SCTM_OK;
    for (int i = 0; i < count; ++i) {
        if (status) status[i] = st[i];
        if (it_done) it_done[i] = it[i];
        if (last_dS) last_dS[i] = ds[i];
        if (st[i] != SCTM_OK && st[i] != SCTM_ENOCONV && worst == SCTM_OK) worst = (sctm_status)st[i];
    }
    if (worst != SCTM_OK) return worst;
    for (int i = 0; i < count; ++i)
        if (st[i] == SCTM_ENOCONV) return SCTM_ENOCONV;
    return SCTM_OK;
}

sctm_status sctm_autotune_info(sctm_ctx* ctx, int network, int* emu, int* eligible) {
    API_BEGIN(ctx)
    if (network < 0 || network > 1) throw Error(SCTM_EINVAL, "bad network");
    if (emu) *emu = ctx->net[network].tuned_emu;
    if (eligible) *eligible = ctx->net[network].tuned_total;
    return SCTM_OK;
    API_END(ctx)
}

size_t sctm_device_bytes(const sctm_ctx* ctx) { return ctx && ctx->eng ? ctx->eng->bytes : 0; }

sctm_status sctm_set_profiling(sctm_ctx* ctx, int on) {
    API_BEGIN(ctx)
    if (on < 0 || on > 2) throw Error(SCTM_EINVAL, "profiling mode must be 0, 1 or 2");
    cuda_ok(cudaStreamSynchronize(ctx->eng->stream), "profiling switch");
    ctx->eng->harvest();
    ctx->eng->profile = on != 0;
    ctx->eng->serial = on == 2;
    return SCTM_OK;
    API_END(ctx)
}

sctm_status sctm_profile(sctm_ctx* ctx, double* ctr_ms, long long* ctr_launches,
                         long long* ctr_flops, double* svd_ms, long long* svd_calls,
                         long long* kernel_launches, int reset) {
    API_BEGIN(ctx)
    Engine& e = *ctx->eng;
    e.harvest();
    if (ctr_ms) *ctr_ms = e.ctr_ms;
    if (ctr_launches) *ctr_launches = e.ctr_launches;
    if (ctr_flops) *ctr_flops = e.ctr_flops;
    if (svd_ms) *svd_ms = e.svd_ms;
    if (svd_calls) *svd_calls = e.svd_calls;
    if (kernel_launches) *kernel_launches = e.kernel_launches.load();
    if (reset) {
        e.ctr_ms = e.svd_ms = 0;
        e.ctr_launches = e.ctr_flops = e.svd_calls = 0;
        for (int i = 0; i < Engine::kKernels; ++i) {
            e.kern_ms[i] = 0;
            e.kern_launches[i] = e.kern_flops[i] = e.kern_bytes[i] = 0;
        }
        e.kernel_launches = 0;
    }
    return SCTM_OK;
    API_END(ctx)
}

}  // extern "C"

// ---------------------------------------------------------------------------------------------
// sctm_gemm: one plain row-major contraction through the library's kernels, in any form
// ---------------------------------------------------------------------------------------------
sctm_status sctm_profile_kernel(sctm_ctx* ctx, int kernel, double* ms, long long* launches,
                                long long* flops, long long* bytes) {
    API_BEGIN(ctx)
    if (kernel < SCTM_KERNEL_F64 || kernel > SCTM_KERNEL_CHOL) throw Error(SCTM_EINVAL, "bad kernel");
    Engine& e = *ctx->eng;
    e.harvest();
    if (ms) *ms = e.kern_ms[kernel];
    if (launches) *launches = e.kern_launches[kernel];
    if (flops) *flops = e.kern_flops[kernel];
    if (bytes) *bytes = e.kern_bytes[kernel];
    return SCTM_OK;
    API_END(ctx)
}

// Device (or managed) memory of device `dev`: memory of another GPU is rejected, since the
// kernels run on the current device and could not reach it without peer access.
static bool on_device(const void* p, int dev) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (at.type == cudaMemoryTypeManaged) return true;
    return at.type == cudaMemoryTypeDevice && at.device == dev;
}

static bool stream_on(cudaStream_t s, int dev) {
    if (s == nullptr || s == cudaStreamLegacy || s == cudaStreamPerThread) return true;
    int sd = -1;
    if (cudaStreamGetDevice(s, &sd) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return sd == dev;
}

// sctm_chol_orth: one Cholesky-QR pass of the partial SVD on device buffers, either kernel
sctm_status sctm_chol_orth(const double* G, int k, double shift, double* T, int variant,
                           void* cuda_stream) {
    if (!G || !T || k < 1 || k > kPsvdMaxK || !(shift >= 0.0)) return SCTM_EINVAL;
    if (variant != SCTM_CHOL_CTA && variant != SCTM_CHOL_CLUSTER) return SCTM_EINVAL;
    if (variant == SCTM_CHOL_CLUSTER && !chol_cluster_fits(k)) return SCTM_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SCTM_ECUDA;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    if (!on_device(G, dev) || !on_device(T, dev) || !stream_on(s, dev)) return SCTM_EINVAL;
    double* Xg = nullptr;
    if (variant == SCTM_CHOL_CTA && k > kPsvdSmemK &&
        cudaMalloc((void**)&Xg, (size_t)k * k * sizeof(double)) != cudaSuccess)
        return SCTM_ENOMEM;
    if (variant == SCTM_CHOL_CLUSTER)
        launch_chol_orth_cluster(G, k, shift, T, s);
    else
        launch_chol_orth_cta(G, k, shift, T, Xg, s);
    sctm_status st = SCTM_OK;
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
        st = SCTM_ECUDA;
    if (Xg) cudaFree(Xg);
    return st;
}

// sctm_jacobi_svd: the partial SVD's k x k Jacobi SVD on device buffers, either kernel
sctm_status sctm_jacobi_svd(const double* B, int k, double* S, double* U, double* W, int variant,
                            void* cuda_stream) {
    if (!B || !S || !U || !W || k < 1 || k > kPsvdMaxK) return SCTM_EINVAL;
    if (variant != SCTM_JACOBI_CTA && variant != SCTM_JACOBI_CLUSTER) return SCTM_EINVAL;
    if (variant == SCTM_JACOBI_CLUSTER && !jacobi_cluster_fits(k)) return SCTM_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SCTM_ECUDA;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    if (!on_device(B, dev) || !on_device(S, dev) || !on_device(U, dev) || !on_device(W, dev) ||
        !stream_on(s, dev))
        return SCTM_EINVAL;
    const int kp = k + (k & 1);
    int* info = nullptr;
    double* Vg = nullptr;
    if (cudaMalloc((void**)&info, sizeof(int)) != cudaSuccess) return SCTM_ENOMEM;
    sctm_status st = SCTM_OK;
    if (variant == SCTM_JACOBI_CTA && k > kPsvdSmemK &&
        cudaMalloc((void**)&Vg, (size_t)kp * (kp + 1) * sizeof(double)) != cudaSuccess)
        st = SCTM_ENOMEM;
    int info_host = 0;
    if (st == SCTM_OK && cudaMemsetAsync(info, 0, sizeof(int), s) != cudaSuccess) st = SCTM_ECUDA;
    if (st == SCTM_OK) {
        if (variant == SCTM_JACOBI_CLUSTER)
            launch_jacobi_svd_cluster(B, k, S, U, W, info, s);
        else
            launch_jacobi_svd_cta(B, k, S, U, W, info, Vg, s);
        if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
            st = SCTM_ECUDA;
        else if (cudaMemcpy(&info_host, info, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
            st = SCTM_ECUDA;
        else if (info_host)
            st = SCTM_ECUSOLVER;
    }
    cudaFree(info);
    if (Vg) cudaFree(Vg);
    return st;
}

sctm_status sctm_gemm(const double* X, const double* Y, double* O, int M, int N, int K,
                      int precision, void* cuda_stream) {
    if (!X || !Y || !O || M < 1 || N < 1 || K < 1) return SCTM_EINVAL;
    if (precision < SCTM_PREC_FP64 || precision > SCTM_PREC_F64EMU) return SCTM_EINVAL;
    if ((long long)M * K >= (1LL << 31) || (long long)K * N >= (1LL << 31) ||
        (long long)M * N >= (1LL << 31))
        return SCTM_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SCTM_ECUDA;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    if (!on_device(X, dev) || !on_device(Y, dev) || !on_device(O, dev) || !stream_on(s, dev))
        return SCTM_EINVAL;
    std::vector<int> xm(M), xk(K), yk(K), yn(N), om(M), on(N);
    for (int m = 0; m < M; ++m) xm[m] = m * K, om[m] = m * N;
    for (int k = 0; k < K; ++k) xk[k] = k, yk[k] = k * N;
    for (int n = 0; n < N; ++n) yn[n] = n, on[n] = n;
    CtrLaunch a;
    a.X = X;
    a.Y = Y;
    a.O = O;
    a.M = M;
    a.N = N;
    a.K = K;
    a.precision = precision;
    // the engine's split-K rule, for the kernel this precision runs on
    const bool tc = precision != SCTM_PREC_FP64;
    const int bm = tc ? 128 : 64, bn = 64, align = tc ? 32 : 16;
    const long long tiles = (long long)((M + bm - 1) / bm) * ((N + bn - 1) / bn);
    int splits = 1, kchunk = K;
    if (tiles < 152 && K > 256) {
        int want = (int)std::min<long long>(std::max<long long>(304 / tiles, 1), (K + 127) / 128);
        want = std::max(1, std::min(want, 128));
        int kc = (K + want - 1) / want;
        kc = ((kc + align - 1) / align) * align;
        if ((K + kc - 1) / kc > 1) {
            splits = (K + kc - 1) / kc;
            kchunk = kc;
        }
    }
    a.tile = 64;
    a.splits = a.tc_splits = splits;
    a.kchunk = a.tc_kchunk = kchunk;
    // test switch: the first bounded wait of each tensor-core CTA gives up at once
    if (const char* tw = getenv("SCTM_TEST_FIRST_WAIT_ZERO"))
        if (tw[0] == '1') a.first_wait_limit = 0;
    std::vector<void*> bufs;
    auto dev_copy = [&](const std::vector<int>& v) -> int* {
        void* p = nullptr;
        if (cudaMalloc(&p, v.size() * sizeof(int)) != cudaSuccess) return nullptr;
        bufs.push_back(p);
        if (cudaMemcpy(p, v.data(), v.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess)
            return nullptr;
        return (int*)p;
    };
    sctm_status st = SCTM_OK;
    int err_host = 0;
    a.xm = dev_copy(xm);
    a.xk = dev_copy(xk);
    a.yk = dev_copy(yk);
    a.yn = dev_copy(yn);
    a.om = dev_copy(om);
    a.on = dev_copy(on);
    a.err = dev_copy({0});
    if (!a.xm || !a.xk || !a.yk || !a.yn || !a.om || !a.on || !a.err) st = SCTM_ENOMEM;
    if (st == SCTM_OK && precision != SCTM_PREC_FP64) {
        void* p = nullptr;
        if (cudaMalloc(&p, 2 * kScaleBlocks * sizeof(double)) != cudaSuccess)
            st = SCTM_ENOMEM;
        else
            bufs.push_back(p), a.scale_ws = (double*)p;
        void* q = nullptr;
        const size_t bx = std::max(tc_pack_bytes_x(a), emu_pack_bytes_x(a));
        const size_t by = std::max(tc_pack_bytes_y(a), emu_pack_bytes_y(a));
        if (st == SCTM_OK && cudaMalloc(&q, bx) != cudaSuccess)
            st = SCTM_ENOMEM;
        else if (st == SCTM_OK)
            bufs.push_back(q), a.pack_x = q;
        q = nullptr;
        if (st == SCTM_OK && cudaMalloc(&q, by) != cudaSuccess)
            st = SCTM_ENOMEM;
        else if (st == SCTM_OK)
            bufs.push_back(q), a.pack_y = q;
        q = nullptr;
        if (st == SCTM_OK && cudaMalloc(&q, emu_exp_ints(a) * sizeof(int)) != cudaSuccess)
            st = SCTM_ENOMEM;
        else if (st == SCTM_OK)
            bufs.push_back(q), a.rexp = (int*)q;
    }
    if (st == SCTM_OK && splits > 1) {
        void* p = nullptr;
        if (cudaMalloc(&p, (size_t)splits * M * N * sizeof(double)) != cudaSuccess)
            st = SCTM_ENOMEM;
        else
            bufs.push_back(p), a.partial = (double*)p;
    }
    if (st == SCTM_OK) {
        launch_ctr(a, s);
        if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
            st = SCTM_ECUDA;
        else if (cudaMemcpy(&err_host, a.err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
            st = SCTM_ECUDA;
        else if (err_host)
            st = SCTM_ETIMEOUT;
    }
    cudaGetLastError();
    for (void* p : bufs) cudaFree(p);
    return st;
}
