// Reverse mode of the split-CTMRG plans and the fixed-point adjoint.
//
// The paper's gradient (Sec. II, Eq. "gradient expression") treats the converged environment as
// fixed.  The derivative of the converged free energy itself, d f / d A, also carries the
// environment's dependence on A.  With E* = F(E*, A) the fixed point of one iteration F (the
// left, right, up and down moves of Sec. III.B, each ending with the Frobenius normalisation) and
// ln kappa(E, A) the per-site value of Sec. II,
//     d ln kappa / d A = d ln kappa / d A |_E + lambda^T dF/dA,   (I - J^T) lambda = w,
// J = dF/dE at E*, w = (d ln kappa / d E)^T (implicit differentiation of the fixed point).
//
// Every plan records a tape while it is built: its contractions, its projector pairs (one unit
// each: M = rho_B rho_T, SVD, sign gauge, P_B = rho_T V S^-1/2, P_T = S^-1/2 U^T rho_B), the
// final normalisation and ln kappa.  The backward plans are built from the tapes in reverse: a
// contraction O = X Y gives dX += dO Y^T and dY += X^T dO as contractions of the same kernels
// (accumulating), the projector pair the backward of a truncated SVD computed from the full
// singular basis, the normalisation y = x / |x| gives dx = (dy - y <y, dy>) / |x|.
//
// Checkpointed recompute: one more forward iteration at E*, with full SVDs, keeps every
// intermediate of the four moves in the plans' own buffers, and each move's input environment
// is copied to a snapshot before the move (the moves overwrite it); the backward of move m reads
// the snapshot of its input.  The linear system for lambda is solved by restarted GMRES, each
// matrix-vector product one backward iteration (down, up, right, left); the fixed-point
// iteration has a slowly decaying, nearly gauge-like mode, which GMRES handles in far fewer
// products than the plain iteration lambda <- w + J^T lambda.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <unordered_set>

#include "engine.h"

namespace sctm {

#define ADJ_CUDA(x)                                                                           \
    do {                                                                                      \
        cudaError_t e_ = (x);                                                                 \
        if (e_ != cudaSuccess) throw Error(SCTM_ECUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
    } while (0)

// ---------------------------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------------------------
struct ZeroItem {
    double* p;
    long long n;
};

__global__ void adj_zero_kernel(const ZeroItem* items, int count) {
    for (int i = blockIdx.y; i < count; i += gridDim.y) {
        const ZeroItem it = items[i];
        for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < it.n;
             j += (long long)gridDim.x * blockDim.x)
            it.p[j] = 0.0;
    }
}

// dst[i][c] = src[i][c] scale[c]  (rows x k, row-major)
__global__ void adj_scale_cols_kernel(const double* src, const double* scale, long long rows, int k,
                                      double* dst) {
    const long long total = rows * k;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x)
        dst[e] = src[e] * scale[e % k];
}

// dst[c][j] = src[c][j] scale[c]  (k x cols, row-major)
__global__ void adj_scale_rows_kernel(const double* src, const double* scale, int k, long long cols,
                                      double* dst) {
    const long long total = (long long)k * cols;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x)
        dst[e] = src[e] * scale[e / cols];
}

__device__ double adj_block_sum(double v) {
    __shared__ double ws[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) ws[w] = v;
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    double t = threadIdx.x < nw ? ws[threadIdx.x] : 0.0;
    if (w == 0)
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    __shared__ double res;
    if (threadIdx.x == 0) res = t;
    __syncthreads();
    const double out = res;
    __syncthreads();
    return out;
}

// dS[c] = d/ds_c of <dPB, PB> + <dPT, PT> through scale[c] = s_c^-1/2:
// -1/2 scale[c]^2 (sum_i PB[i][c] dPB[i][c] + sum_j PT[c][j] dPT[c][j]); 0 where scale is 0
// (a cut-off singular value leaves the projectors unchanged).  One block per column c.
__global__ void adj_proj_ds_kernel(const double* PB, const double* dPB, long long rows,
                                   const double* PT, const double* dPT, long long cols,
                                   const double* scale, int k, double* dS) {
    const int c = blockIdx.x;
    double v = 0.0;
    for (long long i = threadIdx.x; i < rows; i += blockDim.x) v += PB[i * k + c] * dPB[i * k + c];
    for (long long j = threadIdx.x; j < cols; j += blockDim.x)
        v += PT[(long long)c * cols + j] * dPT[(long long)c * cols + j];
    v = adj_block_sum(v);
    if (threadIdx.x == 0) {
        const double sc = scale[c];
        dS[c] = -0.5 * sc * sc * v;
    }
}

// The full right singular basis as columns (n x n, column-major): column c is Vcols[:, c] for
// c < kc (the columns the sign gauge acted on), else row c of V^T.
__global__ void adj_assemble_v_kernel(const double* Vcols, const double* VT, int n, int kc,
                                      double* V) {
    const long long total = (long long)n * n;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(e % n), c = (int)(e / n);
        V[e] = (c < kc && Vcols) ? Vcols[(long long)c * n + r] : VT[c + (long long)r * n];
    }
}

// Core of the SVD backward for M = U S V^T (square, full basis), gradients dU, dV on the first k
// columns and dS on the first k values (J = U^T dU, K = V^T dV given as n x k, column-major):
//   C_ij = F_ij (J_ij - J_ji) s_j + s_i F_ij (K_ij - K_ji) + delta_ij dS_i,
//   F_ij = (s_j^2 - s_i^2) / ((s_j^2 - s_i^2)^2 + eta)   (i != j; a Lorentzian broadening of
// 1 / (s_j^2 - s_i^2) for near-degenerate pairs, eta = (eps s_0^2)^2), and dM = U C V^T.  Pairs
// of discarded values (i, j >= k) have J_ij = J_ji = 0.
__global__ void adj_svd_core_kernel(const double* Jk, const double* Kk, const double* S,
                                    const double* dS, int n, int k, double eps, double degen,
                                    double* C) {
    const double s0sq = S[0] * S[0];
    const double eta = (eps * s0sq) * (eps * s0sq);
    const double dtol = degen * S[0];
    const long long total = (long long)n * n;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e % n), j = (int)(e / n);
        double v = 0.0;
        if (i == j) {
            v = i < k ? dS[i] : 0.0;
        } else if (i < k || j < k) {
            const double Jij = j < k ? Jk[i + (long long)j * n] : 0.0;
            const double Jji = i < k ? Jk[j + (long long)i * n] : 0.0;
            const double Kij = j < k ? Kk[i + (long long)j * n] : 0.0;
            const double Kji = i < k ? Kk[j + (long long)i * n] : 0.0;
            const double si = S[i], sj = S[j];
            const double d = sj * sj - si * si;
            // pairs closer than degen s_0 are treated as degenerate: a rotation inside their
            // subspace changes no gauge-invariant result, so it carries no gradient
            const double F = fabs(sj - si) <= dtol ? 0.0 : d / (d * d + eta);
            v = F * (Jij - Jji) * sj + si * F * (Kij - Kji);
        }
        C[e] = v;
    }
}

// Backward of the Frobenius normalisation y = x / |x| written through a strided view:
// dx += (dy - x <x, dy> / |x|^2) / |x|.  One block per item.
struct NormBwdItem {
    const double* src;   // x, contiguous
    double* dsrc;        // dx, contiguous (accumulated)
    const double* ddst;  // dy, read through the destination view's strides
    int d0, d1, d2;
    long long s0, s1, s2;
};

__global__ void adj_norm_bwd_kernel(const NormBwdItem* items) {
    const NormBwdItem it = items[blockIdx.x];
    const long long n = (long long)it.d0 * it.d1 * it.d2;
    double ss = 0.0, xd = 0.0;
    for (long long i = threadIdx.x; i < n; i += blockDim.x) {
        const int i2 = (int)(i % it.d2);
        const long long r = i / it.d2;
        const int i1 = (int)(r % it.d1), i0 = (int)(r / it.d1);
        const double x = it.src[i], dy = it.ddst[i0 * it.s0 + i1 * it.s1 + i2 * it.s2];
        ss += x * x;
        xd += x * dy;
    }
    ss = adj_block_sum(ss);
    xd = adj_block_sum(xd);
    if (!(ss > 0.0)) return;
    const double nrm = sqrt(ss), a = xd / ss;
    for (long long i = threadIdx.x; i < n; i += blockDim.x) {
        const int i2 = (int)(i % it.d2);
        const long long r = i / it.d2;
        const int i1 = (int)(r % it.d1), i0 = (int)(r / it.d1);
        const double dy = it.ddst[i0 * it.s0 + i1 * it.s1 + i2 * it.s2];
        it.dsrc[i] += (dy - it.src[i] * a) / nrm;
    }
}

// Backward pseudo-inverse scales: scale[c] where s_c >= gcut s_0, else 0.  Kept singular
// values below gcut s_0 are held fixed in the backward: their projector columns are
// rounding-level directions whose exact sensitivities (through s^-1/2 and 1 / (s_j^2 - s_i^2))
// are huge and cancel in any gauge-invariant result, but make the adjoint's linear system
// numerically useless.
__global__ void adj_gcut_kernel(const double* S, const double* scale, int k, double gcut,
                                double* out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < k) out[c] = S[c] >= gcut * S[0] ? scale[c] : 0.0;
}

// d ln kappa / d Z for ln kappa = ln Z11 + ln Z00 - ln Z10 - ln Z01
__global__ void adj_lnk_seed_kernel(const double* z00, const double* z10, const double* z01,
                                    const double* z11, double* g00, double* g10, double* g01,
                                    double* g11) {
    g00[0] = 1.0 / z00[0];
    g10[0] = -1.0 / z10[0];
    g01[0] = -1.0 / z01[0];
    g11[0] = 1.0 / z11[0];
}

// fixed-order dot product of two flat vectors: one block, out[0] = sum_i a[i] b[i]
__global__ void adj_dot_kernel(const double* a, const double* b, long long n, double* out) {
    double v = 0.0;
    for (long long i = threadIdx.x; i < n; i += blockDim.x) v = fma(a[i], b[i], v);
    v = adj_block_sum(v);
    if (threadIdx.x == 0) out[0] = v;
}

// y = alpha x + beta y
__global__ void adj_axpby_kernel(double alpha, const double* x, double beta, double* y, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        y[i] = alpha * x[i] + beta * y[i];
}

// d f / d A = -T (d ln kappa_num / dA - d ln kappa_den / dA)
__global__ void adj_combine_kernel(const double* a, const double* b, double T, int n, double* g) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) g[i] = -T * (a[i] - b[i]);
}

void launch_adj_combine(const double* dnum, const double* dden, double T, int n, double* g,
                        cudaStream_t s) {
    adj_combine_kernel<<<(n + 255) / 256, 256, 0, s>>>(dnum, dden, T, n, g);
}

static int blocks_for(long long n) {
    return (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, 2048));
}

// ---------------------------------------------------------------------------------------------
// backward plans
// ---------------------------------------------------------------------------------------------
struct Adjoint {
    std::unordered_map<const double*, double*> grad;      // forward buffer -> its gradient
    std::unordered_map<const double*, double*> snap[4];   // stored tensor -> move m's input copy
    Plan bwd_move[4], bwd_local;
    const double* env_base[16] = {nullptr};
    long long env_n[16] = {0};
    long long n_env = 0;
    double* dA = nullptr;       // gradient of the site tensor A (both the ket and the bra slot)
    double* dA_local = nullptr;
    double* w = nullptr;        // d ln kappa / d E, flat
    double* x = nullptr;        // lambda, flat
    double* r = nullptr;        // residual / scratch, flat
    double* z = nullptr;
    std::vector<double*> V;     // Krylov basis
    double* red = nullptr;      // one device double for reductions
};

Network::Network() = default;
Network::~Network() {
    if (graph_exec) cudaGraphExecDestroy(graph_exec);
    if (graph) cudaGraphDestroy(graph);
}

namespace {

constexpr int kKrylov = 40;          // GMRES restart length
constexpr double kBroadening = 1e-12;  // SVD backward: Lorentzian width, relative to s_0^2
constexpr double kDegenerate = 0.0;    // SVD backward: |s_i - s_j| <= this s_0 counts as degenerate

struct FnStepA : Step {
    std::function<void(cudaStream_t)> f;
    explicit FnStepA(std::function<void(cudaStream_t)> g) : f(std::move(g)) {}
    void run(Engine& e) override {
        f(e.strm(sid));
        e.kernel_launches += 1;
    }
};

Ten with_base(const Ten& t, double* p) {
    Ten o = t;
    o.p = p;
    return o;
}

Ten mat(double* p, int rows, int cols) {  // column-major rows x cols
    Ten t;
    t.p = p;
    t.nd = 2;
    t.dim[0] = rows;
    t.dim[1] = cols;
    t.st[0] = 1;
    t.st[1] = rows;
    return t;
}

// [r..., c] view of a column-major n x n (or n x k) matrix whose row index is the row-major
// multi-index over rdims
Ten cols_view(double* p, const Ten& like_r, int nr_dims, int n, int k) {
    Ten t;
    t.p = p;
    t.nd = nr_dims + 1;
    long long s = 1;
    for (int i = nr_dims - 1; i >= 0; --i) {
        t.dim[i] = like_r.dim[i];
        t.st[i] = s;
        s *= like_r.dim[i];
    }
    t.dim[nr_dims] = k;
    t.st[nr_dims] = n;
    return t;
}

class Builder {
public:
    Builder(Engine& e, Network& net, Adjoint& ad) : e_(e), net_(net), ad_(ad) {
        if (const char* v = getenv("SCTM_ADJ_EPS")) eps_ = atof(v);
        if (const char* v = getenv("SCTM_ADJ_DEGEN")) degen_ = atof(v);
    }

    // Backward plan of one tape.  snap: the move's input snapshots (nullptr for the local plan).
    // The plan first zeroes the gradients of the tape's intermediates.
    void build(const Tape& tape, Plan& P, std::unordered_map<const double*, double*>* snap,
               bool is_move) {
        snap_ = snap;
        zeros_.clear();
        Plan body;
        std::unordered_set<const double*> live;
        for (auto it = tape.rbegin(); it != tape.rend(); ++it) {
            const TapeOp& op = *it;
            switch (op.kind) {
                case TapeOp::LNK: {
                    double* g[4];
                    for (int q = 0; q < 4; ++q) {
                        g[q] = grad_of(op.z[q], 1);
                        live.insert(op.z[q]);
                    }
                    const double *z0 = op.z[0], *z1 = op.z[1], *z2 = op.z[2], *z3 = op.z[3];
                    push(body, [=](cudaStream_t s) {
                        adj_lnk_seed_kernel<<<1, 1, 0, s>>>(z0, z1, z2, z3, g[0], g[1], g[2], g[3]);
                    });
                    break;
                }
                case TapeOp::NORM: {
                    std::vector<NormBwdItem> items;
                    std::vector<ZeroItem> clear;
                    for (const auto& pr : op.items) {
                        const Ten& src = pr.first;
                        const Ten& dst = pr.second;
                        NormBwdItem b;
                        b.src = src.p;
                        b.dsrc = grad_of(src.p, src.numel());
                        b.ddst = grad_of(dst.p, dst.numel());
                        b.d0 = src.dim[0];
                        b.d1 = src.nd > 1 ? src.dim[1] : 1;
                        b.d2 = src.nd > 2 ? src.dim[2] : 1;
                        b.s0 = dst.st[0];
                        b.s1 = dst.nd > 1 ? dst.st[1] : 0;
                        b.s2 = dst.nd > 2 ? dst.st[2] : 0;
                        items.push_back(b);
                        clear.push_back({grad_of(dst.p, dst.numel()), dst.numel()});
                        live.insert(src.p);
                    }
                    NormBwdItem* dev = (NormBwdItem*)e_.dalloc(
                        (long long)(items.size() * sizeof(NormBwdItem) + 7) / 8);
                    if (!e_.dry)
                        ADJ_CUDA(cudaMemcpy(dev, items.data(), items.size() * sizeof(NormBwdItem),
                                            cudaMemcpyHostToDevice));
                    const int cnt = (int)items.size();
                    push(body, [=](cudaStream_t s) { adj_norm_bwd_kernel<<<cnt, 1024, 0, s>>>(dev); });
                    // the move overwrote these stored tensors: their incoming gradient is consumed
                    push_zero(body, clear);
                    break;
                }
                case TapeOp::CTR: {
                    if (!live.count(op.O.p)) break;
                    const std::string& spec = op.spec;
                    const size_t comma = spec.find(','), arrow = spec.find("->");
                    const std::string xl = spec.substr(0, comma),
                                      yl = spec.substr(comma + 1, arrow - comma - 1),
                                      ol = spec.substr(arrow + 2);
                    const Ten dO = gradT(op.O);
                    if (needs_grad(op.X.p)) {
                        const Ten dX = gradT(op.X);
                        e_.ctr(net_, body, ol + "," + yl + "->" + xl, dO, fwd(op.Y), &dX, nullptr,
                               nullptr, true);
                        live.insert(op.X.p);
                    }
                    if (needs_grad(op.Y.p)) {
                        const Ten dY = gradT(op.Y);
                        e_.ctr(net_, body, xl + "," + ol + "->" + yl, fwd(op.X), dO, &dY, nullptr,
                               nullptr, true);
                        live.insert(op.Y.p);
                    }
                    break;
                }
                case TapeOp::PROJ: {
                    if (!live.count(op.PB.p) && !live.count(op.PT.p)) break;
                    proj_backward(op, body);
                    live.insert(op.X.p);
                    live.insert(op.Y.p);
                    break;
                }
            }
        }
        // zero this plan's intermediate gradients first, then run the body
        (void)is_move;
        push_zero(P, zeros_);
        for (auto& st : body) P.push_back(std::move(st));
    }

    double* grad_of(const double* base, long long min_n) {
        auto it = ad_.grad.find(base);
        if (it != ad_.grad.end()) return it->second;
        long long n = e_.size_of(base);
        if (n <= 0) n = min_n;
        if (n < min_n) throw Error(SCTM_EINVAL, "adjoint: gradient buffer smaller than its view");
        double* g = e_.dalloc(n);
        ad_.grad[base] = g;
        if (!is_env(base) && base != net_.A.p) zeros_.push_back({g, n});
        return g;
    }

private:
    Engine& e_;
    Network& net_;
    Adjoint& ad_;
    std::unordered_map<const double*, double*>* snap_ = nullptr;
    std::vector<ZeroItem> zeros_;
    double eps_ = kBroadening, degen_ = kDegenerate;

    bool is_env(const double* p) const {
        for (int q = 0; q < 16; ++q)
            if (ad_.env_base[q] == p) return true;
        return false;
    }
    bool needs_grad(const double* p) const { return e_.dry || p != net_.O.p; }
    Ten gradT(const Ten& t) { return with_base(t, grad_of(t.p, 1)); }
    Ten fwd(const Ten& t) const {
        if (snap_) {
            auto it = snap_->find(t.p);
            if (it != snap_->end()) return with_base(t, it->second);
        }
        return t;
    }

    void push(Plan& P, std::function<void(cudaStream_t)> f) {
        auto st = std::make_unique<FnStepA>(std::move(f));
        st->sid = 0;
        P.push_back(std::move(st));
    }

    void push_zero(Plan& P, const std::vector<ZeroItem>& list) {
        if (list.empty()) return;
        ZeroItem* dev = (ZeroItem*)e_.dalloc((long long)(list.size() * sizeof(ZeroItem) + 7) / 8);
        if (!e_.dry)
            ADJ_CUDA(cudaMemcpy(dev, list.data(), list.size() * sizeof(ZeroItem),
                                cudaMemcpyHostToDevice));
        const int cnt = (int)list.size();
        push(P, [=](cudaStream_t s) {
            adj_zero_kernel<<<dim3(64, std::min(cnt, 1024)), 256, 0, s>>>(dev, cnt);
        });
    }

    // Backward of one projector pair (see the file comment), from dP_B and dP_T.
    void proj_backward(const TapeOp& op, Plan& P) {
        const int n = op.n, k = op.chi;
        const char K = '#';
        const std::string &labels = op.spec, &tl = op.tl, &rl = op.rl, &rlL = op.rlL,
                          &Llab = op.Llab;
        const int nr = (int)rl.size();
        const Ten& U = op.X;
        const Ten& L = op.Y;
        const Ten gPB = gradT(op.PB), gPT = gradT(op.PT);
        const long long rowsB = op.PB.numel() / k, colsT = op.PT.numel() / k;
        double* dPBs = e_.dalloc(op.PB.numel());
        double* dPTs = e_.dalloc(op.PT.numel());
        double* dS = e_.dalloc(k);
        double* Vfull = (op.vt || op.kc < n) ? e_.dalloc((long long)n * n) : op.Vcols;
        double* dUk = e_.dalloc((long long)n * k);
        double* dVk = e_.dalloc((long long)n * k);
        double* Jk = e_.dalloc((long long)n * k);
        double* Kk = e_.dalloc((long long)n * k);
        double* Cm = e_.dalloc((long long)n * n);
        double* T1 = e_.dalloc((long long)n * n);
        double* scale = e_.dalloc(k);
        const double *S0 = op.S, *scale_f = op.scale;
        const Network* np = &net_;  // the cutoff is read at launch time (sctm_set_grad_mode)
        const double *PBp = op.PB.p, *PTp = op.PT.p, *gPBp = gPB.p, *gPTp = gPT.p;
        push(P, [=](cudaStream_t s) {
            adj_gcut_kernel<<<(k + 127) / 128, 128, 0, s>>>(S0, scale_f, k, np->adj_gcut, scale);
            adj_scale_cols_kernel<<<blocks_for(rowsB * k), 256, 0, s>>>(gPBp, scale, rowsB, k, dPBs);
            adj_scale_rows_kernel<<<blocks_for(colsT * k), 256, 0, s>>>(gPTp, scale, k, colsT, dPTs);
            adj_proj_ds_kernel<<<k, 256, 0, s>>>(PBp, gPBp, rowsB, PTp, gPTp, colsT, scale, k, dS);
        });
        if (Vfull != op.Vcols) {
            const double *Vc = op.Vcols, *VT = op.VT;
            const int kc = op.kc;
            push(P, [=](cudaStream_t s) {
                adj_assemble_v_kernel<<<blocks_for((long long)n * n), 256, 0, s>>>(Vc, VT, n, kc, Vfull);
            });
        }
        // views: [tl..., K] of dP_B, [K, tl...] of dP_T, [r..., K] of the singular vectors
        const Ten vPBs = with_base(op.PB, dPBs), vPTs = with_base(op.PT, dPTs);
        Ten rlike;  // the remaining legs' dimensions, in order
        rlike.nd = nr;
        for (int i = 0, j = 0; i < U.nd; ++i)
            if (tl.find(labels[i]) == std::string::npos) rlike.dim[j++] = U.dim[i];
        const Ten Vk = cols_view(Vfull, rlike, nr, n, k);
        const Ten Ukv = cols_view(op.Us, rlike, nr, n, k);
        const Ten dVkv = cols_view(dVk, rlike, nr, n, k);
        const Ten dUkv = cols_view(dUk, rlike, nr, n, k);
        const Ten dU = gradT(U), dL = gradT(L);
        const std::string tK = tl + K, Kt = std::string(1, K) + tl;
        // through P_B = U V S^-1/2 and P_T = S^-1/2 U_s^T L
        e_.ctr(net_, P, tK + "," + rl + K + "->" + labels, vPBs, Vk, &dU, nullptr, nullptr, true);
        e_.ctr(net_, P, labels + "," + tK + "->" + rl + K, U, vPBs, &dVkv);
        e_.ctr(net_, P, Kt + "," + rlL + K + "->" + Llab, vPTs, Ukv, &dL, nullptr, nullptr, true);
        e_.ctr(net_, P, Kt + "," + Llab + "->" + rlL + K, vPTs, L, &dUkv);
        // SVD backward: J = U^T dU_k, K = V^T dV_k, C (core), dM = U C V^T
        const Ten Um = mat(op.Us, n, n), Vm = mat(Vfull, n, n);
        const Ten dUm = mat(dUk, n, k), dVm = mat(dVk, n, k), Jm = mat(Jk, n, k), Km = mat(Kk, n, k);
        e_.ctr(net_, P, "ai,ac->ic", Um, dUm, &Jm);
        e_.ctr(net_, P, "ai,ac->ic", Vm, dVm, &Km);
        const double* S = op.S;
        const double eps = eps_, degen = degen_;
        push(P, [=](cudaStream_t s) {
            adj_svd_core_kernel<<<blocks_for((long long)n * n), 256, 0, s>>>(Jk, Kk, S, dS, n, k,
                                                                              eps, degen, Cm);
        });
        const Ten Cmat = mat(Cm, n, n), T1m = mat(T1, n, n);
        const Ten gM = gradT(op.M);
        const Ten gMm = mat(gM.p, n, n);
        e_.ctr(net_, P, "ab,bc->ac", Um, Cmat, &T1m);
        e_.ctr(net_, P, "ac,dc->ad", T1m, Vm, &gMm);
        // through M = L^T U (contracted over the truncated legs)
        e_.ctr(net_, P, rlL + rl + "," + labels + "->" + Llab, gM, U, &dL, nullptr, nullptr, true);
        e_.ctr(net_, P, Llab + "," + rlL + rl + "->" + labels, L, gM, &dU, nullptr, nullptr, true);
    }
};

}  // namespace

// ---------------------------------------------------------------------------------------------
// driver
// ---------------------------------------------------------------------------------------------
void Engine::build_adjoint(Network& net) {
    Engine& e = *this;
    net.adj.reset(new Adjoint());
    Adjoint& ad = *net.adj;
    const size_t first = net.ctr_steps.size();
    int q = 0;
    for (int i = 0; i < 4; ++i) ad.env_base[q] = net.C[i].p, ad.env_n[q++] = net.C[i].numel();
    for (int i = 0; i < 4; ++i)
        for (int x = 0; x < 3; ++x) ad.env_base[q] = net.T[i][x].p, ad.env_n[q++] = net.T[i][x].numel();
    ad.n_env = 0;
    for (int i = 0; i < 16; ++i) {
        ad.grad[ad.env_base[i]] = e.dalloc(ad.env_n[i]);
        ad.n_env += ad.env_n[i];
        for (int m = 0; m < 4; ++m) ad.snap[m][ad.env_base[i]] = e.dalloc(ad.env_n[i]);
    }
    ad.dA = e.dalloc(net.A.numel());
    ad.grad[net.A.p] = ad.dA;
    ad.dA_local = e.dalloc(net.A.numel());
    Builder b(e, net, ad);
    const int saved_stream = e.cur_stream;
    e.cur_stream = 0;
    for (int m = 0; m < 4; ++m) b.build(net.tape_move[m], ad.bwd_move[m], &ad.snap[m], true);
    b.build(net.tape_local, ad.bwd_local, nullptr, false);
    e.cur_stream = saved_stream;
    e.assign_workspace(net, first);
    ad.w = e.dalloc(ad.n_env);
    ad.x = e.dalloc(ad.n_env);
    ad.r = e.dalloc(ad.n_env);
    ad.z = e.dalloc(ad.n_env);
    for (int i = 0; i <= kKrylov; ++i) ad.V.push_back(e.dalloc(ad.n_env));
    ad.red = e.dalloc(1);
}

namespace {

struct Solver {
    Engine& e;
    Network& net;
    Adjoint& ad;
    cudaStream_t s;
    int matvecs = 0;

    void gather(double* flat) {  // env gradients -> flat vector
        long long off = 0;
        for (int q = 0; q < 16; ++q) {
            ADJ_CUDA(cudaMemcpyAsync(flat + off, ad.grad[ad.env_base[q]], ad.env_n[q] * sizeof(double),
                                     cudaMemcpyDeviceToDevice, s));
            off += ad.env_n[q];
        }
    }
    void scatter(const double* flat) {
        long long off = 0;
        for (int q = 0; q < 16; ++q) {
            ADJ_CUDA(cudaMemcpyAsync(ad.grad[ad.env_base[q]], flat + off, ad.env_n[q] * sizeof(double),
                                     cudaMemcpyDeviceToDevice, s));
            off += ad.env_n[q];
        }
    }
    void zero_env_grads() {
        for (int q = 0; q < 16; ++q)
            ADJ_CUDA(cudaMemsetAsync(ad.grad[ad.env_base[q]], 0, ad.env_n[q] * sizeof(double), s));
    }
    double dot(const double* a, const double* b) {
        adj_dot_kernel<<<1, 1024, 0, s>>>(a, b, ad.n_env, ad.red);
        double h = 0.0;
        ADJ_CUDA(cudaMemcpyAsync(&h, ad.red, sizeof(double), cudaMemcpyDeviceToHost, s));
        ADJ_CUDA(cudaStreamSynchronize(s));
        return h;
    }
    void axpby(double a, const double* x, double b, double* y) {
        adj_axpby_kernel<<<blocks_for(ad.n_env), 256, 0, s>>>(a, x, b, y, ad.n_env);
    }
    // out = (I - J^T) v; the A-gradient of J_A^T v is left in ad.dA
    bool debug = false;
    void apply(const double* v, double* out) {
        scatter(v);
        ADJ_CUDA(cudaMemsetAsync(ad.dA, 0, net.A.numel() * sizeof(double), s));
        for (int m = 3; m >= 0; --m) e.run(ad.bwd_move[m]);
        gather(out);
        if (debug) {  // SCTM_ADJ_DEBUG=1: |J^T v| / |v| of every product
            const double nv = std::sqrt(dot(v, v)), nj = std::sqrt(dot(out, out));
            fprintf(stderr, "adjoint d=%d product %d: |J^T v|/|v| = %.3e\n", net.d, matvecs,
                    nv > 0 ? nj / nv : 0.0);
        }
        axpby(1.0, v, -1.0, out);
        ++matvecs;
    }
};

}  // namespace

void Engine::adjoint_lnk_grad(Network& net, double* dA_out, double tol, int max_mv, int* mv_used,
                              double* residual) {
    if (dry) throw Error(SCTM_EINVAL, "adjoint in a dry run");
    if (!net.adj) build_adjoint(net);
    Adjoint& ad = *net.adj;
    const int saved_lane = cur_lane;
    cur_lane = 0;
    const bool saved_serial = serial;
    cudaStream_t s = lanes[0].streams[0];
    // checkpointed recompute: one iteration at the fixed point with full SVDs, each move's input
    // environment saved first; then the local contractions at the resulting environment
    force_full_svd = true;
    try {
        for (int m = 0; m < 4; ++m) {
            for (int q = 0; q < 16; ++q)
                ADJ_CUDA(cudaMemcpyAsync(ad.snap[m][ad.env_base[q]], ad.env_base[q],
                                         ad.env_n[q] * sizeof(double), cudaMemcpyDeviceToDevice, s));
            run(net.move[m]);
        }
    } catch (...) {
        force_full_svd = false;
        cur_lane = saved_lane;
        throw;
    }
    force_full_svd = false;
    serial = true;  // the backward plans write shared gradient buffers: one stream
    Solver sv{*this, net, ad, s};
    if (const char* dbg = getenv("SCTM_ADJ_DEBUG")) sv.debug = dbg[0] == '1';
    try {
        run(net.local);
        sv.zero_env_grads();
        ADJ_CUDA(cudaMemsetAsync(ad.dA, 0, net.A.numel() * sizeof(double), s));
        run(ad.bwd_local);
        sv.gather(ad.w);
        ADJ_CUDA(cudaMemcpyAsync(ad.dA_local, ad.dA, net.A.numel() * sizeof(double),
                                 cudaMemcpyDeviceToDevice, s));
        // restarted GMRES for (I - J^T) x = w, x0 = 0
        const double wn = std::sqrt(std::max(sv.dot(ad.w, ad.w), 0.0));
        ADJ_CUDA(cudaMemsetAsync(ad.x, 0, ad.n_env * sizeof(double), s));
        double rel = wn > 0.0 ? 1.0 : 0.0;
        if (wn > 0.0) {
            ADJ_CUDA(cudaMemcpyAsync(ad.r, ad.w, ad.n_env * sizeof(double), cudaMemcpyDeviceToDevice, s));
            double beta = wn;
            while (rel > tol && sv.matvecs < max_mv) {
                const int m = kKrylov;
                std::vector<double> H((m + 1) * m, 0.0), cs(m, 0.0), sn(m, 0.0), g(m + 1, 0.0);
                g[0] = beta;
                sv.axpby(1.0 / beta, ad.r, 0.0, ad.V[0]);
                int j = 0;
                for (; j < m && sv.matvecs < max_mv; ++j) {
                    sv.apply(ad.V[j], ad.z);
                    for (int i = 0; i <= j; ++i) {  // modified Gram-Schmidt
                        const double h = sv.dot(ad.z, ad.V[i]);
                        H[i * m + j] = h;
                        sv.axpby(-h, ad.V[i], 1.0, ad.z);
                    }
                    const double hn = std::sqrt(std::max(sv.dot(ad.z, ad.z), 0.0));
                    H[(j + 1) * m + j] = hn;
                    if (hn > 0.0) sv.axpby(1.0 / hn, ad.z, 0.0, ad.V[j + 1]);
                    for (int i = 0; i < j; ++i) {  // previous Givens rotations
                        const double a = H[i * m + j], b = H[(i + 1) * m + j];
                        H[i * m + j] = cs[i] * a + sn[i] * b;
                        H[(i + 1) * m + j] = -sn[i] * a + cs[i] * b;
                    }
                    const double a = H[j * m + j], b = H[(j + 1) * m + j];
                    const double rr = std::hypot(a, b);
                    cs[j] = rr > 0.0 ? a / rr : 1.0;
                    sn[j] = rr > 0.0 ? b / rr : 0.0;
                    H[j * m + j] = rr;
                    H[(j + 1) * m + j] = 0.0;
                    g[j + 1] = -sn[j] * g[j];
                    g[j] = cs[j] * g[j];
                    rel = std::fabs(g[j + 1]) / wn;
                    if (sv.debug) fprintf(stderr, "adjoint d=%d GMRES step %d: rel %.3e\n", net.d, j, rel);
                    if (rel <= tol || hn == 0.0) {
                        ++j;
                        break;
                    }
                }
                // x += V y, H y = g (upper triangular j x j)
                std::vector<double> y(j, 0.0);
                for (int i = j - 1; i >= 0; --i) {
                    double t = g[i];
                    for (int l = i + 1; l < j; ++l) t -= H[i * m + l] * y[l];
                    y[i] = H[i * m + i] != 0.0 ? t / H[i * m + i] : 0.0;
                }
                for (int i = 0; i < j; ++i) sv.axpby(y[i], ad.V[i], 1.0, ad.x);
                if (rel <= tol || sv.matvecs >= max_mv) break;
                // true residual for the restart: r = w - (I - J^T) x
                sv.apply(ad.x, ad.r);
                sv.axpby(1.0, ad.w, -1.0, ad.r);
                beta = std::sqrt(std::max(sv.dot(ad.r, ad.r), 0.0));
                rel = beta / wn;
                if (beta == 0.0) break;
            }
        }
        // dA = d ln kappa / dA |_E + J_A^T x
        sv.scatter(ad.x);
        ADJ_CUDA(cudaMemsetAsync(ad.dA, 0, net.A.numel() * sizeof(double), s));
        for (int m = 3; m >= 0; --m) run(ad.bwd_move[m]);
        adj_axpby_kernel<<<blocks_for(net.A.numel()), 256, 0, s>>>(1.0, ad.dA_local, 1.0, ad.dA,
                                                                  net.A.numel());
        ADJ_CUDA(cudaMemcpyAsync(dA_out, ad.dA, net.A.numel() * sizeof(double),
                                 cudaMemcpyDeviceToDevice, s));
        ADJ_CUDA(cudaStreamSynchronize(s));
        ADJ_CUDA(cudaGetLastError());
        if (mv_used) *mv_used = sv.matvecs;
        if (residual) *residual = rel;
    } catch (...) {
        serial = saved_serial;
        cur_lane = saved_lane;
        throw;
    }
    serial = saved_serial;
    cur_lane = saved_lane;
}

}  // namespace sctm
