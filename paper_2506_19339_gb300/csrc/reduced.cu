// The reduced method on the GPU (Sec. II, Fig. 3; the comparison method of Sec. IV.A): the
// physical legs of A, O and A-bar are contracted first into one single-layer tensor
//     a[(ua,uo,ub), (la,lo,lb), (da,do,db), (ra,ro,rb)] = sum_{s,t} A[s,..] O[t,s,..] A-bar[t,..]
// of bond m = D d D, which standard directional CTMRG then contracts: one corner and one edge
// tensor per side, one projector pair per move from the two-by-two patch around the truncated
// bond (rho_T and rho_B the upper and lower halves, M = rho_B rho_T over the truncated legs, the
// projectors of Eqs. "projector construction" / "projector construction 2").  Its leading cost is
// O(chi^3 D^6 d^3) against the split method's O(chi^3 D^3 d^3) (Sec. III.C).
//
// The plans reuse the split method's machinery: the einsum contraction builder (gather tables,
// no transpose kernels), the projector builder (every SVD mode), the Frobenius normalisation,
// the convergence spectrum and ln kappa.  The edge tensors live in the T[i][0] slots (leg m); the
// int and bra slots are empty.  The cold start is the reduced oracle's: C = e_0 e_0^T and
// T[0][0][:] = 1.
#include <algorithm>
#include <cstring>

#include "engine.h"

namespace sctm {

#define RED_CUDA(x)                                                                           \
    do {                                                                                      \
        cudaError_t e_ = (x);                                                                 \
        if (e_ != cudaSuccess) throw Error(SCTM_ECUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
    } while (0)

namespace {

struct FnStepR : Step {
    std::function<void(cudaStream_t)> f;
    explicit FnStepR(std::function<void(cudaStream_t)> g) : f(std::move(g)) {}
    void run(Engine& e) override {
        f(e.strm(sid));
        e.kernel_launches += 1;
    }
};

struct RFrame {
    Ten C[4];
    Ten T[4];
    Ten a;
};

// the right, up and down moves are the left move in a relabelled network: up = reflection about
// the diagonal, right = rotation by 180 degrees, down = both (a single layer needs no exchange
// of ket and bra)
RFrame rframe(const Network& n, const Ten& a, int move) {
    RFrame f;
    auto tr = [](const Ten& t) { return permute(t, {1, 0}); };
    auto sw = [](const Ten& t) { return permute(t, {1, 0, 2}); };
    if (move == SCTM_MOVE_LEFT) {
        for (int i = 0; i < 4; ++i) f.C[i] = n.C[i], f.T[i] = n.T[i][0];
        f.a = a;
    } else if (move == SCTM_MOVE_UP) {
        f.C[0] = tr(n.C[0]);
        f.C[1] = tr(n.C[3]);
        f.C[2] = tr(n.C[2]);
        f.C[3] = tr(n.C[1]);
        f.T[0] = n.T[3][0];
        f.T[1] = n.T[2][0];
        f.T[2] = n.T[1][0];
        f.T[3] = n.T[0][0];
        f.a = permute(a, {1, 0, 3, 2});
    } else if (move == SCTM_MOVE_RIGHT) {
        f.C[0] = n.C[2];
        f.C[1] = n.C[3];
        f.C[2] = n.C[0];
        f.C[3] = n.C[1];
        f.T[0] = sw(n.T[2][0]);
        f.T[1] = sw(n.T[3][0]);
        f.T[2] = sw(n.T[0][0]);
        f.T[3] = sw(n.T[1][0]);
        f.a = permute(a, {2, 3, 0, 1});
    } else {  // down: the diagonal reflection of the rotated frame
        RFrame r = rframe(n, a, SCTM_MOVE_RIGHT);
        f.C[0] = tr(r.C[0]);
        f.C[1] = tr(r.C[3]);
        f.C[2] = tr(r.C[2]);
        f.C[3] = tr(r.C[1]);
        f.T[0] = r.T[3];
        f.T[1] = r.T[2];
        f.T[2] = r.T[1];
        f.T[3] = r.T[0];
        f.a = permute(r.a, {1, 0, 3, 2});
    }
    return f;
}

}  // namespace

void Engine::build_reduced_network(Network& net) {
    const int chi = net.chi, D = net.D, d = net.d, p = net.p, m = D * d * D;
    for (int i = 0; i < 4; ++i) {
        net.C[i] = alloc({chi, chi});
        net.T[i][0] = alloc({chi, chi, m});
        net.T[i][1] = view(dalloc(1), {0});
        net.T[i][2] = view(dalloc(1), {0});
    }
    net.S_old = dalloc(chi);
    net.dS = dalloc(1);
    net.lnk = dalloc(2);
    net.E = alloc({p, D, D, D, D});
    // the fused site tensor, rebuilt whenever A changes (net.site)
    double* abuf = dalloc((long long)m * m * m * m);
    const Ten a12 = view(abuf, {D, d, D, D, d, D, D, d, D, D, d, D});
    const Ten a = view(abuf, {m, m, m, m});
    net.fused = a;
    {
        Plan& P = net.site;
        const Ten X = ctr(net, P, "sabcd,tsefgh->tabcdefgh", net.A, net.O);
        ctr(net, P, "tabcdefgh,tijkl->aeibfjcgkdhl", X, net.B, &a12);
    }
    // the four directional moves
    for (int mv = 0; mv < 4; ++mv) {
        Plan& P = net.move[mv];
        const RFrame f = rframe(net, a, mv);
        auto C = [&](const char* spec, const Ten& X, const Ten& Y) { return ctr(net, P, spec, X, Y); };
        const Ten &C1 = f.C[0], &C2 = f.C[1], &C3 = f.C[2], &C4 = f.C[3];
        const Ten &T1 = f.T[0], &T2 = f.T[1], &T3 = f.T[2], &T4 = f.T[3], &A1 = f.a;
        // quarters of the two-by-two patch around the bond between the two rows of the column
        const Ten C1T1 = C("av,ahu->vhu", C1, T1);
        const Ten Q1 = C("huxl,ulDr->xDhr", C("vhu,vxl->huxl", C1T1, T4), A1);   // [xl, a.d | h, a.r]
        const Ten Q2 = C("Huyr,ulDr->HlDy", C("Hhu,hyr->Huyr", T1, C("hw,wyr->hyr", C2, T2)), A1);
        const Ten C4T3 = C("av,ahd->vhd", C4, T3);
        const Ten Q4 = C("hdxl,uldr->xuhr", C("vhd,xvl->hdxl", C4T3, T4), A1);   // [xl, a.u | h, a.r]
        const Ten Q3 = C("Hdyr,uldr->Hluy", C("Hhd,hyr->Hdyr", T3, C("hw,ywr->hyr", C3, T2)), A1);
        const Ten Rt = C("xDhr,hrEy->xDEy", Q1, Q2);   // upper half [xl, a.d | E, xr]
        const Ten Rb = C("xuhr,hrEy->xuEy", Q4, Q3);   // lower half
        const PPair pp = projector(net, P, Rt, Rb, "xDEy", "xD");   // P_B [x, D, k], P_T [k, x, D]
        const Ten C1n = C("vhu,kvu->hk", C1T1, pp.PT);
        const Ten C4n = C("vhd,vdk->hk", C4T3, pp.PB);
        const Ten T4n = C("KXDr,kXD->Kkr", C("uKXl,ulDr->KXDr", C("xuK,xXl->uKXl", pp.PB, T4), A1),
                          pp.PT);
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
        items.push_back(item(T4n, f.T[3]));
        items.push_back(item(C4n, f.C[3]));
        NormItem* dev = (NormItem*)dalloc((long long)(items.size() * sizeof(NormItem) + 7) / 8);
        if (!dry)
            RED_CUDA(cudaMemcpy(dev, items.data(), items.size() * sizeof(NormItem),
                                cudaMemcpyHostToDevice));
        const int cnt = (int)items.size();
        push(P, std::make_unique<FnStepR>([=](cudaStream_t s) { launch_normalize(dev, cnt, s); }));
    }
    build_spectrum(*this, net);
    // local contractions (Sec. II, Fig. 4(b), (c)) of the single-layer network
    {
        Plan& P = net.local;
        auto C = [&](const char* spec, const Ten& X, const Ten& Y, const Ten* out = nullptr) {
            return ctr(net, P, spec, X, Y, out);
        };
        const Ten &C1 = net.C[0], &C2 = net.C[1], &C3 = net.C[2], &C4 = net.C[3];
        const Ten &T1 = net.T[0][0], &T2 = net.T[1][0], &T3 = net.T[2][0], &T4 = net.T[3][0];
        const Ten Z00 = C("vw,vw->", C("hv,hw->vw", C1, C2), C("hv,hw->vw", C4, C3));
        const Ten top = C("vhu,hw->vuw", C("av,ahu->vhu", C1, T1), C2);   // [v1, a.u, v2]
        const Ten bot = C("vhd,hw->vdw", C("av,ahd->vhd", C4, T3), C3);
        const Ten Z10 = C("vuw,vuw->", top, bot);
        const Ten lft = C("hxl,gx->hlg", C("hv,vxl->hxl", C1, T4), C4);
        const Ten rgt = C("hyl,gy->hlg", C("hw,wyl->hyl", C2, T2), C3);
        const Ten Z01 = C("hlg,hlg->", lft, rgt);
        Ten X = C("vuw,vxl->uwxl", top, T4);
        X = C("uwxl,ulDr->wxDr", X, a);
        X = C("wxDr,wyr->xDy", X, T2);
        const Ten Z11 = C("xDy,xDy->", X, bot);
        // the bra environment: Z11 with A-bar removed, the fused legs split back into (A, O, A-bar)
        const Ten top6 = view(top.p, {chi, D, d, D, chi});
        const Ten bot6 = view(bot.p, {chi, D, d, D, chi});
        const Ten T4v = view(T4.p, {chi, chi, D, d, D});
        const Ten T2v = view(T2.p, {chi, chi, D, d, D});
        X = C("vpoqw,vxlLM->poqwxlLM", top6, T4v);
        X = C("poqwxlLM,splEr->oqwxLMsEr", X, net.A);
        X = C("oqwxLMsEr,tsoLfR->qwxMErtfR", X, net.O);
        X = C("qwxMErtfR,wyrRS->qxMEtfyS", X, T2v);
        C("qxMEtfyS,xEfgy->tqMgS", X, bot6, &net.E);
        double *z00 = Z00.p, *z10 = Z10.p, *z01 = Z01.p, *z11 = Z11.p, *lnk = net.lnk;
        net.z[0] = z00;
        net.z[1] = z10;
        net.z[2] = z01;
        net.z[3] = z11;
        push(P, std::make_unique<FnStepR>(
                    [=](cudaStream_t s) { launch_lnkappa(z00, z10, z01, z11, lnk, s); }));
    }
    finalize(net);
    set_precision(net, SCTM_PREC_FP64);
}

// The reduced oracle's cold start: every C = e_0 e_0^T, every T with T[0][0][:] = 1.
void Engine::init_reduced_env(Network& net) {
    cold_svd(net);
    if (dry) return;
    RED_CUDA(cudaMemsetAsync(dev_err, 0, 2 * sizeof(int), stream));
    const int chi = net.chi;
    const long long m = net.T[0][0].dim[2];
    std::vector<double> c((size_t)chi * chi, 0.0), t((size_t)chi * chi * m, 0.0);
    c[0] = 1.0;
    for (long long j = 0; j < m; ++j) t[(size_t)j] = 1.0;
    for (int i = 0; i < 4; ++i) {
        RED_CUDA(cudaMemcpyAsync(net.C[i].p, c.data(), c.size() * sizeof(double),
                                 cudaMemcpyHostToDevice, stream));
        RED_CUDA(cudaMemcpyAsync(net.T[i][0].p, t.data(), t.size() * sizeof(double),
                                 cudaMemcpyHostToDevice, stream));
    }
    launch_zero(net.S_old, net.chi, stream);
    RED_CUDA(cudaStreamSynchronize(stream));  // the host vectors go out of scope
}

}  // namespace sctm
