// C-ABI of libtdgrad and the host-side planner: basis upload, Schwarz
// factors, pair screening and class sort, quartet tiles, class launches and
// the final reduction.  Every arithmetic step of the gradient runs in the
// CUDA kernels; the host only orders work and moves buffers.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "class_launchers.cuh"
#include "setup_kernels.cuh"

using namespace tg;

namespace {

struct DevArena {
    char *p = nullptr;
    size_t cap = 0;
    size_t used = 0;
    cudaError_t reserve(size_t bytes)
    {
        if (bytes <= cap) return cudaSuccess;
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
        cudaError_t e = cudaMalloc(&p, bytes);
        if (e == cudaSuccess) cap = bytes;
        return e;
    }
    template <typename T>
    T *take(size_t n)
    {
        size_t off = (used + 255) & ~(size_t)255;
        used = off + n * sizeof(T);
        return reinterpret_cast<T *>(p + off);
    }
    void release()
    {
        if (p) cudaFree(p);
        p = nullptr;
        cap = used = 0;
    }
};

inline size_t al(size_t bytes) { return (bytes + 255) & ~(size_t)255; }

}  // namespace

struct tg_basis {
    int device = 0;
    int natom = 0, nshell = 0, nbf = 0, nprim = 0;
    std::vector<int> sh_atom, sh_l, sh_nprim, sh_poff, sh_bf;
    double *d_xyz = nullptr, *d_exps = nullptr, *d_coefs = nullptr, *d_cn = nullptr, *d_boys = nullptr;
    int *d_sh_atom = nullptr, *d_sh_l = nullptr, *d_sh_nprim = nullptr, *d_sh_poff = nullptr, *d_sh_bf = nullptr;
    std::vector<double> Q, Qd;  // per canonical pair key (x >= y)
    double Qmax = 0.0, Qdmax = 0.0;
    DevArena ws;
    int nsm = 0;
};

namespace {

#define TG_CUDA(call)                      \
    do {                                   \
        cudaError_t e_ = (call);           \
        if (e_ != cudaSuccess) {           \
            cudaGetLastError();            \
            return e_ == cudaErrorMemoryAllocation ? TG_ENOMEM : TG_ECUDA; \
        }                                  \
    } while (0)

inline long long pkey(int x, int y)
{
    const int X = x > y ? x : y, Y = x > y ? y : x;
    return (long long)X * (X + 1) / 2 + Y;
}

void free_basis(tg_basis *b)
{
    if (!b) return;
    cudaFree(b->d_xyz);
    cudaFree(b->d_exps);
    cudaFree(b->d_coefs);
    cudaFree(b->d_cn);
    cudaFree(b->d_boys);
    cudaFree(b->d_sh_atom);
    cudaFree(b->d_sh_l);
    cudaFree(b->d_sh_nprim);
    cudaFree(b->d_sh_poff);
    cudaFree(b->d_sh_bf);
    b->ws.release();
}

int basis_setup(tg_basis *b, const double *xyz, const double *exps, const double *coefs)
{
    TG_CUDA(cudaGetDevice(&b->device));
    TG_CUDA(cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, b->device));
    const int ns = b->nshell, np = b->nprim;
    TG_CUDA(cudaMalloc(&b->d_xyz, sizeof(double) * 3 * b->natom));
    TG_CUDA(cudaMalloc(&b->d_exps, sizeof(double) * np));
    TG_CUDA(cudaMalloc(&b->d_coefs, sizeof(double) * np));
    TG_CUDA(cudaMalloc(&b->d_cn, sizeof(double) * np));
    TG_CUDA(cudaMalloc(&b->d_boys, sizeof(double) * BOYS_NG * (BOYS_M + 1)));
    TG_CUDA(cudaMalloc(&b->d_sh_atom, sizeof(int) * ns));
    TG_CUDA(cudaMalloc(&b->d_sh_l, sizeof(int) * ns));
    TG_CUDA(cudaMalloc(&b->d_sh_nprim, sizeof(int) * ns));
    TG_CUDA(cudaMalloc(&b->d_sh_poff, sizeof(int) * ns));
    TG_CUDA(cudaMalloc(&b->d_sh_bf, sizeof(int) * ns));
    TG_CUDA(cudaMemcpy(b->d_xyz, xyz, sizeof(double) * 3 * b->natom, cudaMemcpyHostToDevice));
    TG_CUDA(cudaMemcpy(b->d_exps, exps, sizeof(double) * np, cudaMemcpyHostToDevice));
    TG_CUDA(cudaMemcpy(b->d_coefs, coefs, sizeof(double) * np, cudaMemcpyHostToDevice));
    TG_CUDA(cudaMemcpy(b->d_sh_atom, b->sh_atom.data(), sizeof(int) * ns, cudaMemcpyHostToDevice));
    TG_CUDA(cudaMemcpy(b->d_sh_l, b->sh_l.data(), sizeof(int) * ns, cudaMemcpyHostToDevice));
    TG_CUDA(cudaMemcpy(b->d_sh_nprim, b->sh_nprim.data(), sizeof(int) * ns, cudaMemcpyHostToDevice));
    TG_CUDA(cudaMemcpy(b->d_sh_poff, b->sh_poff.data(), sizeof(int) * ns, cudaMemcpyHostToDevice));
    TG_CUDA(cudaMemcpy(b->d_sh_bf, b->sh_bf.data(), sizeof(int) * ns, cudaMemcpyHostToDevice));
    k_boys_table<<<(BOYS_NG + 127) / 128, 128>>>(b->d_boys);
    k_normalise<<<(ns + 127) / 128, 128>>>(ns, b->d_sh_l, b->d_sh_nprim, b->d_sh_poff, b->d_exps, b->d_coefs, b->d_cn);
    TG_CUDA(cudaGetLastError());
    // Schwarz factors of every canonical shell pair (geometry only, cached)
    const long long npr = (long long)ns * (ns + 1) / 2;
    std::vector<int2> prs((size_t)npr);
    for (int x = 0; x < ns; ++x)
        for (int y = 0; y <= x; ++y) prs[(size_t)pkey(x, y)] = make_int2(x, y);
    int2 *d_prs = nullptr;
    double *d_Q = nullptr, *d_Qd = nullptr;
    cudaError_t e = cudaMalloc(&d_prs, sizeof(int2) * npr);
    if (e == cudaSuccess) e = cudaMalloc(&d_Q, sizeof(double) * npr);
    if (e == cudaSuccess) e = cudaMalloc(&d_Qd, sizeof(double) * npr);
    if (e == cudaSuccess) e = cudaMemcpy(d_prs, prs.data(), sizeof(int2) * npr, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        k_schwarz<<<(unsigned)((npr + 127) / 128), 128>>>((int)npr, d_prs, b->d_xyz, b->d_sh_atom, b->d_sh_l,
                                                          b->d_sh_nprim, b->d_sh_poff, b->d_exps, b->d_cn, d_Q, d_Qd);
        e = cudaGetLastError();
    }
    b->Q.resize((size_t)npr);
    b->Qd.resize((size_t)npr);
    if (e == cudaSuccess) e = cudaMemcpy(b->Q.data(), d_Q, sizeof(double) * npr, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(b->Qd.data(), d_Qd, sizeof(double) * npr, cudaMemcpyDeviceToHost);
    cudaFree(d_prs);
    cudaFree(d_Q);
    cudaFree(d_Qd);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? TG_ENOMEM : TG_ECUDA;
    }
    for (long long k = 0; k < npr; ++k) {
        b->Qmax = std::max(b->Qmax, b->Q[(size_t)k]);
        b->Qdmax = std::max(b->Qdmax, b->Qd[(size_t)k]);
    }
    return TG_OK;
}

struct HostPair {
    int sa, sb, np, key;
    double Q, Qd;
};

}  // namespace

extern "C" {

void tg_options_default(tg_options *o)
{
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->screen_tol = 1e-10;
    o->precision = TG_FP64;
    o->router = nullptr;
    o->mixed_tol = 1e-6;
    o->device_ptrs = 0;
    o->stream = nullptr;
    o->rank = 0;
    o->nranks = 1;
    o->timing = 0;
}

const char *tg_strerror(int s)
{
    switch (s) {
    case TG_OK: return "ok";
    case TG_EINVAL: return "invalid argument";
    case TG_EUNSUPPORTED: return "unsupported input (l > 2, several lr omegas, too many pairs)";
    case TG_ENOMEM: return "out of memory";
    case TG_ECUDA: return "CUDA runtime error";
    case TG_ETIMEOUT: return "bounded device wait expired";
    case TG_EROUTER: return "router missing or malformed";
    default: return "unknown status";
    }
}

int tg_basis_create(int natom, const double *xyz, int nshell, const int *shell_atom, const int *shell_l,
                    const int *shell_nprim, const double *exps, const double *coefs, tg_basis **out)
{
    if (!out) return TG_EINVAL;
    *out = nullptr;
    if (natom < 1 || nshell < 1 || !xyz || !shell_atom || !shell_l || !shell_nprim || !exps || !coefs)
        return TG_EINVAL;
    for (int i = 0; i < 3 * natom; ++i)
        if (!std::isfinite(xyz[i])) return TG_EINVAL;
    long long nprim = 0, nbf = 0;
    for (int s = 0; s < nshell; ++s) {
        if (shell_atom[s] < 0 || shell_atom[s] >= natom) return TG_EINVAL;
        if (shell_nprim[s] < 1 || shell_nprim[s] > 16) return TG_EINVAL;
        if (shell_l[s] < 0) return TG_EINVAL;
        if (shell_l[s] > MAXL) return TG_EUNSUPPORTED;
        nprim += shell_nprim[s];
        nbf += ncart(shell_l[s]);
    }
    if ((long long)nshell * (nshell + 1) / 2 > 0x7fffffffLL) return TG_EUNSUPPORTED;
    for (long long k = 0; k < nprim; ++k)
        if (!(exps[k] > 0.0) || !std::isfinite(exps[k]) || !std::isfinite(coefs[k])) return TG_EINVAL;
    tg_basis *b = new (std::nothrow) tg_basis();
    if (!b) return TG_ENOMEM;
    b->natom = natom;
    b->nshell = nshell;
    b->nprim = (int)nprim;
    b->nbf = (int)nbf;
    b->sh_atom.assign(shell_atom, shell_atom + nshell);
    b->sh_l.assign(shell_l, shell_l + nshell);
    b->sh_nprim.assign(shell_nprim, shell_nprim + nshell);
    b->sh_poff.resize(nshell);
    b->sh_bf.resize(nshell);
    int po = 0, bo = 0;
    for (int s = 0; s < nshell; ++s) {
        b->sh_poff[s] = po;
        b->sh_bf[s] = bo;
        po += shell_nprim[s];
        bo += ncart(shell_l[s]);
    }
    int rc = basis_setup(b, xyz, exps, coefs);
    if (rc != TG_OK) {
        free_basis(b);
        delete b;
        return rc;
    }
    *out = b;
    return TG_OK;
}

int tg_basis_nbf(const tg_basis *b) { return b ? b->nbf : TG_EINVAL; }
int tg_basis_natom(const tg_basis *b) { return b ? b->natom : TG_EINVAL; }

void tg_basis_destroy(tg_basis *b)
{
    if (!b) return;
    free_basis(b);
    delete b;
}

int tg_grad2e(const tg_basis *cb, int npair, const tg_pair *pairs, const tg_options *opt_in, double *grad,
              tg_stats *stats)
{
    auto t0 = std::chrono::steady_clock::now();
    tg_basis *b = const_cast<tg_basis *>(cb);
    if (!b || !pairs || !grad) return TG_EINVAL;
    tg_options opt;
    if (opt_in) opt = *opt_in;
    else tg_options_default(&opt);
    if (npair < 1) return TG_EINVAL;
    if (npair > TG_MAX_PAIRS) return TG_EUNSUPPORTED;
    if (!(opt.screen_tol >= 0.0) || !std::isfinite(opt.screen_tol)) return TG_EINVAL;
    if (opt.nranks < 1 || opt.rank < 0 || opt.rank >= opt.nranks) return TG_EINVAL;
    if (opt.precision != TG_FP64 && opt.precision != TG_MIXED_BOUND && opt.precision != TG_MIXED_LEARNED)
        return TG_EINVAL;
    if (opt.precision != TG_FP64) return TG_EUNSUPPORTED;
    double omega = 0.0;
    int use_lr = 0;
    for (int p = 0; p < npair; ++p) {
        const tg_pair &q = pairs[p];
        if (!q.A || !q.B) return TG_EINVAL;
        if (!std::isfinite(q.c_J) || !std::isfinite(q.c_K) || !std::isfinite(q.c_K_lr) || std::isnan(q.omega))
            return TG_EINVAL;
        if (q.c_K_lr != 0.0 && q.omega > 0.0) {
            if (use_lr && q.omega != omega) return TG_EUNSUPPORTED;
            use_lr = 1;
            omega = q.omega;
        }
    }
    cudaStream_t st = (cudaStream_t)opt.stream;
    const int nbf = b->nbf, ns = b->nshell, natom = b->natom;
    const size_t nbf2 = (size_t)nbf * nbf;
    TG_CUDA(cudaSetDevice(b->device));

    // ---- pass 1: densities, symmetrised copies, block maxima
    DevArena &W = b->ws;
    const int nmat_up = opt.device_ptrs ? 0 : 2 * npair;
    size_t need1 = al(sizeof(double) * nbf2) * (nmat_up + 2 * npair) + al(sizeof(double) * (size_t)ns * ns) +
                   al(sizeof(double) * ns) + al(sizeof(double) * TG_MAX_PAIRS) + al(sizeof(double) * 3 * natom) +
                   al(sizeof(unsigned long long) * 3 * NQC) + 4096;
    // pass-2 sizes are not known yet; reserve pass 1 now and grow below
    DensArgs den;
    std::memset(&den, 0, sizeof(den));
    den.npair = npair;
    den.nbf = nbf;
    den.use_lr = use_lr;
    den.omega = omega;
    for (int p = 0; p < npair; ++p) {
        den.cJ[p] = pairs[p].c_J;
        den.cK[p] = pairs[p].c_K;
        den.cKlr[p] = (pairs[p].omega > 0.0) ? pairs[p].c_K_lr : 0.0;
    }

    // ---- host pair screening needs Mmax; compute it after upload.  To keep
    // one arena, the arena is sized for pass 1 plus the largest possible pass 2
    // (all candidate pairs kept) on first use.
    const long long npr_all = (long long)ns * (ns + 1) / 2;

    W.used = 0;
    TG_CUDA(W.reserve(need1));
    double *dmat[2 * TG_MAX_PAIRS];
    for (int k = 0; k < nmat_up; ++k) dmat[k] = W.take<double>(nbf2);
    double *dS[2 * TG_MAX_PAIRS];
    for (int k = 0; k < 2 * npair; ++k) dS[k] = W.take<double>(nbf2);
    double *dM = W.take<double>((size_t)ns * ns);
    double *dMrow = W.take<double>(ns);
    double *dw = W.take<double>(TG_MAX_PAIRS);
    double *dgrad = W.take<double>(3 * natom);
    unsigned long long *dcnt = W.take<unsigned long long>(3 * NQC);
    const size_t pass1_used = W.used;

    for (int p = 0; p < npair; ++p) {
        if (opt.device_ptrs) {
            den.A[p] = pairs[p].A;
            den.B[p] = pairs[p].B;
        } else {
            TG_CUDA(cudaMemcpyAsync(dmat[2 * p], pairs[p].A, sizeof(double) * nbf2, cudaMemcpyHostToDevice, st));
            TG_CUDA(cudaMemcpyAsync(dmat[2 * p + 1], pairs[p].B, sizeof(double) * nbf2, cudaMemcpyHostToDevice, st));
            den.A[p] = dmat[2 * p];
            den.B[p] = dmat[2 * p + 1];
        }
        const unsigned gs = (unsigned)((nbf2 + 255) / 256);
        k_symm<<<gs, 256, 0, st>>>(nbf, den.A[p], dS[2 * p]);
        k_symm<<<gs, 256, 0, st>>>(nbf, den.B[p], dS[2 * p + 1]);
        den.S[p] = dS[2 * p];
        den.T[p] = dS[2 * p + 1];
    }
    double hw[TG_MAX_PAIRS];
    for (int p = 0; p < npair; ++p) hw[p] = std::sqrt(std::fabs(den.cJ[p]) + std::fabs(den.cK[p]) + std::fabs(den.cKlr[p]));
    TG_CUDA(cudaMemcpyAsync(dw, hw, sizeof(double) * npair, cudaMemcpyHostToDevice, st));
    {
        const unsigned gs = (unsigned)((npr_all + 127) / 128);
        k_blockmax<<<gs, 128, 0, st>>>(ns, b->d_sh_bf, b->d_sh_l, den, dw, dM, dMrow);
        k_rowmax<<<(ns + 127) / 128, 128, 0, st>>>(ns, dM, dMrow);
        TG_CUDA(cudaGetLastError());
    }
    std::vector<double> Mrow(ns);
    TG_CUDA(cudaMemcpyAsync(Mrow.data(), dMrow, sizeof(double) * ns, cudaMemcpyDeviceToHost, st));
    TG_CUDA(cudaStreamSynchronize(st));
    double Mmax = 0.0;
    for (int x = 0; x < ns; ++x) Mmax = std::max(Mmax, Mrow[x]);

    // ---- pair screening and class sort (Sec. II.C: presort by K and Schwarz bound)
    const double tau = opt.screen_tol;
    const double scale = 8.0 * npair;
    std::vector<HostPair> cls[NPC];
    for (int x = 0; x < ns; ++x)
        for (int y = 0; y <= x; ++y) {
            const long long k = pkey(x, y);
            const double q = b->Q[(size_t)k], qd = b->Qd[(size_t)k];
            if (tau > 0.0) {
                const double bnd = scale * std::max(qd * b->Qmax, q * b->Qdmax) * Mmax * Mmax;
                if (bnd < tau) continue;
            }
            int sa = x, sb = y;
            if (b->sh_l[y] > b->sh_l[x]) std::swap(sa, sb);
            HostPair hp;
            hp.sa = sa;
            hp.sb = sb;
            hp.np = b->sh_nprim[sa] * b->sh_nprim[sb];
            hp.key = (int)k;
            hp.Q = q;
            hp.Qd = qd;
            cls[pair_class(b->sh_l[sa], b->sh_l[sb])].push_back(hp);
        }
    long long npairs_kept = 0, nprimpairs = 0;
    for (int c = 0; c < NPC; ++c) {
        std::sort(cls[c].begin(), cls[c].end(), [](const HostPair &u, const HostPair &v) {
            if (u.np != v.np) return u.np > v.np;
            if (u.Qd != v.Qd) return u.Qd > v.Qd;
            return u.key < v.key;
        });
        npairs_kept += (long long)cls[c].size();
        for (auto &hp : cls[c]) nprimpairs += hp.np;
    }
    // per-tile-block maxima for the tile bounds
    std::vector<int> h_sa, h_sb, h_poff, h_np, h_key;
    std::vector<double> h_Q, h_Qd;
    h_sa.reserve(npairs_kept);
    int cls_off[NPC + 1];
    {
        int po = 0, n = 0;
        for (int c = 0; c < NPC; ++c) {
            cls_off[c] = n;
            for (auto &hp : cls[c]) {
                h_sa.push_back(hp.sa);
                h_sb.push_back(hp.sb);
                h_poff.push_back(po);
                h_np.push_back(hp.np);
                h_key.push_back(hp.key);
                h_Q.push_back(hp.Q);
                h_Qd.push_back(hp.Qd);
                po += hp.np;
                ++n;
            }
        }
        cls_off[NPC] = n;
    }

    // ---- quartet tiles per class, screened by a tile bound, sorted by cost
    struct HostTile {
        unsigned bt, kt;
        long long cost;
    };
    std::vector<uint2> tiles_all;
    long long tile_off[NQC + 1];
    int qc_P[NQC], qc_Q[NQC];
    for (int P = 0; P < NPC; ++P)
        for (int Qc = 0; Qc <= P; ++Qc) {
            qc_P[P * (P + 1) / 2 + Qc] = P;
            qc_Q[P * (P + 1) / 2 + Qc] = Qc;
        }
    auto blockmax = [&](int c, int blk, int bsz, double &q, double &qd, double &m) {
        q = qd = m = 0.0;
        const int lo = blk * bsz, hi = std::min((int)cls[c].size(), lo + bsz);
        for (int i = lo; i < hi; ++i) {
            const HostPair &hp = cls[c][i];
            q = std::max(q, hp.Q);
            qd = std::max(qd, hp.Qd);
            m = std::max(m, std::max(Mrow[hp.sa], Mrow[hp.sb]));
        }
    };
    for (int qc = 0; qc < NQC; ++qc) {
        tile_off[qc] = (long long)tiles_all.size();
        const int P = qc_P[qc], Qc = qc_Q[qc];
        const int nP = (int)cls[P].size(), nQ = (int)cls[Qc].size();
        if (!nP || !nQ) continue;
        const int nbt = (nP + TB - 1) / TB, nkt = (nQ + TK - 1) / TK;
        std::vector<double> bq(nbt), bqd(nbt), bm(nbt), kq(nkt), kqd(nkt), km(nkt);
        for (int i = 0; i < nbt; ++i) blockmax(P, i, TB, bq[i], bqd[i], bm[i]);
        for (int i = 0; i < nkt; ++i) blockmax(Qc, i, TK, kq[i], kqd[i], km[i]);
        std::vector<HostTile> ts;
        for (int bt = 0; bt < nbt; ++bt)
            for (int kt = 0; kt < nkt; ++kt) {
                if (P == Qc && kt * TK > bt * TB + TB - 1) continue;
                if (tau > 0.0) {
                    const double Mt = std::max(bm[bt], km[kt]);
                    const double bnd = scale * std::max(bqd[bt] * kq[kt], bq[bt] * kqd[kt]) * Mt * Mt;
                    if (bnd < tau) continue;
                }
                HostTile t;
                t.bt = bt;
                t.kt = kt;
                t.cost = (long long)cls[P][bt * TB].np * cls[Qc][kt * TK].np;
                ts.push_back(t);
            }
        std::stable_sort(ts.begin(), ts.end(), [](const HostTile &u, const HostTile &v) { return u.cost > v.cost; });
        for (auto &t : ts) tiles_all.push_back(make_uint2(t.bt, t.kt));
    }
    tile_off[NQC] = (long long)tiles_all.size();

    // ---- pass 2 buffers
    const int G = std::max(1, 2 * b->nsm);
    const size_t np_k = (size_t)std::max<long long>(npairs_kept, 1);
    const size_t npp = (size_t)std::max<long long>(nprimpairs, 1);
    size_t need2 = pass1_used + 5 * al(sizeof(int) * np_k) + 2 * al(sizeof(double) * np_k) +
                   6 * al(sizeof(double) * npp) + 6 * al(sizeof(float) * npp) +
                   al(sizeof(uint2) * std::max<size_t>(tiles_all.size(), 1)) + al(sizeof(double) * (size_t)G * 3 * natom) +
                   4096;
    if (need2 > W.cap) {
        // grow and redo pass 1 in the bigger arena (the device copies are cheap)
        TG_CUDA(cudaStreamSynchronize(st));
        W.release();
        TG_CUDA(W.reserve(need2 + need2 / 4));
        return tg_grad2e(cb, npair, pairs, opt_in, grad, stats);
    }
    int *d_sa = W.take<int>(np_k), *d_sb = W.take<int>(np_k), *d_poff = W.take<int>(np_k), *d_np = W.take<int>(np_k),
        *d_key = W.take<int>(np_k);
    double *d_Q = W.take<double>(np_k), *d_Qd = W.take<double>(np_k);
    double *pp_p = W.take<double>(npp), *pp_x = W.take<double>(npp), *pp_y = W.take<double>(npp),
           *pp_z = W.take<double>(npp), *pp_K = W.take<double>(npp), *pp_za = W.take<double>(npp);
    float *fp_p = W.take<float>(npp), *fp_x = W.take<float>(npp), *fp_y = W.take<float>(npp),
          *fp_z = W.take<float>(npp), *fp_K = W.take<float>(npp), *fp_za = W.take<float>(npp);
    uint2 *d_tiles = W.take<uint2>(std::max<size_t>(tiles_all.size(), 1));
    double *d_part = W.take<double>((size_t)G * 3 * natom);

    if (npairs_kept > 0) {
        TG_CUDA(cudaMemcpyAsync(d_sa, h_sa.data(), sizeof(int) * npairs_kept, cudaMemcpyHostToDevice, st));
        TG_CUDA(cudaMemcpyAsync(d_sb, h_sb.data(), sizeof(int) * npairs_kept, cudaMemcpyHostToDevice, st));
        TG_CUDA(cudaMemcpyAsync(d_poff, h_poff.data(), sizeof(int) * npairs_kept, cudaMemcpyHostToDevice, st));
        TG_CUDA(cudaMemcpyAsync(d_np, h_np.data(), sizeof(int) * npairs_kept, cudaMemcpyHostToDevice, st));
        TG_CUDA(cudaMemcpyAsync(d_key, h_key.data(), sizeof(int) * npairs_kept, cudaMemcpyHostToDevice, st));
        TG_CUDA(cudaMemcpyAsync(d_Q, h_Q.data(), sizeof(double) * npairs_kept, cudaMemcpyHostToDevice, st));
        TG_CUDA(cudaMemcpyAsync(d_Qd, h_Qd.data(), sizeof(double) * npairs_kept, cudaMemcpyHostToDevice, st));
        k_prim_pairs<<<(unsigned)((npairs_kept + 127) / 128), 128, 0, st>>>(
            (int)npairs_kept, d_sa, d_sb, d_poff, b->d_xyz, b->d_sh_atom, b->d_sh_nprim, b->d_sh_poff, b->d_exps,
            b->d_cn, pp_p, pp_x, pp_y, pp_z, pp_K, pp_za, fp_p, fp_x, fp_y, fp_z, fp_K, fp_za);
        TG_CUDA(cudaGetLastError());
    }
    if (!tiles_all.empty())
        TG_CUDA(cudaMemcpyAsync(d_tiles, tiles_all.data(), sizeof(uint2) * tiles_all.size(), cudaMemcpyHostToDevice, st));
    TG_CUDA(cudaMemsetAsync(d_part, 0, sizeof(double) * (size_t)G * 3 * natom, st));
    TG_CUDA(cudaMemsetAsync(dcnt, 0, sizeof(unsigned long long) * 3 * NQC, st));

    GeoArgs geo;
    geo.natom = natom;
    geo.nshell = ns;
    geo.xyz = b->d_xyz;
    geo.sh_atom = b->d_sh_atom;
    geo.sh_bf = b->d_sh_bf;
    ScreenArgs scr;
    scr.tau = tau;
    scr.scale = scale;
    scr.M = dM;
    scr.nshell = ns;
    scr.rank = opt.rank;
    scr.nranks = opt.nranks;
    PrimPairs pp;
    pp.p = pp_p;
    pp.Px = pp_x;
    pp.Py = pp_y;
    pp.Pz = pp_z;
    pp.K = pp_K;
    pp.za = pp_za;
    pp.fp = fp_p;
    pp.fPx = fp_x;
    pp.fPy = fp_y;
    pp.fPz = fp_z;
    pp.fK = fp_K;
    pp.fza = fp_za;
    OutArgs out;
    out.partials = d_part;
    out.counters = dcnt;
    const size_t stage = (size_t)TILE * 12 * sizeof(double) + (size_t)TILE * 4 * sizeof(int);
    const size_t sgrad = (size_t)3 * natom * sizeof(double);
    out.use_smem = (stage + sgrad) <= 160 * 1024;
    const size_t smem = stage + (out.use_smem ? sgrad : 0);

    auto mkset = [&](int c) {
        PairSet s;
        const int o = cls_off[c];
        s.n = (int)cls[c].size();
        s.sa = d_sa + o;
        s.sb = d_sb + o;
        s.poff = d_poff + o;
        s.np = d_np + o;
        s.Q = d_Q + o;
        s.Qd = d_Qd + o;
        s.key = d_key + o;
        return s;
    };
    int launches = 2 * npair + 3 + (npairs_kept > 0 ? 1 : 0);
    cudaEvent_t ev[NQC + 1];
    bool timed[NQC];
    const bool timing = opt.timing != 0;
    for (int qc = 0; qc < NQC; ++qc) timed[qc] = false;
    if (timing)
        for (int k = 0; k <= NQC; ++k) TG_CUDA(cudaEventCreate(&ev[k]));
    for (int qc = 0; qc < NQC; ++qc) {
        const long long nt = tile_off[qc + 1] - tile_off[qc];
        if (nt <= 0) continue;
        ClassLaunch cl;
        cl.bra = mkset(qc_P[qc]);
        cl.ket = mkset(qc_Q[qc]);
        cl.same = qc_P[qc] == qc_Q[qc];
        cl.ntiles = nt;
        cl.tiles = d_tiles + tile_off[qc];
        cl.route = nullptr;
        OutArgs o = out;
        o.counters = dcnt + 3 * qc;
        const int grid = (int)std::min<long long>(nt, G);
        if (timing) cudaEventRecord(ev[qc], st);
        cudaError_t e = kClassLaunchers[qc](0, grid, smem, st, geo, den, scr, cl, o, pp, b->d_boys);
        if (timing) {
            cudaEventRecord(ev[NQC], st);
            cudaEventSynchronize(ev[NQC]);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, ev[qc], ev[NQC]);
            if (stats) stats->class_ms[qc] = ms;
            timed[qc] = true;
        }
        if (e != cudaSuccess) {
            cudaGetLastError();
            if (timing)
                for (int k = 0; k <= NQC; ++k) cudaEventDestroy(ev[k]);
            return TG_ECUDA;
        }
        ++launches;
    }
    if (timing)
        for (int k = 0; k <= NQC; ++k) cudaEventDestroy(ev[k]);
    k_reduce<<<(3 * natom + 127) / 128, 128, 0, st>>>(3 * natom, G, d_part, dgrad);
    ++launches;
    TG_CUDA(cudaGetLastError());
    unsigned long long hc[3 * NQC];
    TG_CUDA(cudaMemcpyAsync(hc, dcnt, sizeof(hc), cudaMemcpyDeviceToHost, st));
    if (opt.device_ptrs) {
        TG_CUDA(cudaMemcpyAsync(grad, dgrad, sizeof(double) * 3 * natom, cudaMemcpyDeviceToDevice, st));
    } else {
        TG_CUDA(cudaMemcpyAsync(grad, dgrad, sizeof(double) * 3 * natom, cudaMemcpyDeviceToHost, st));
    }
    TG_CUDA(cudaStreamSynchronize(st));
    if (stats) {
        long long q = 0, pq = 0, q32 = 0;
        for (int qc = 0; qc < NQC; ++qc) {
            stats->class_quartets[qc] = (long long)hc[3 * qc];
            stats->class_prim_quartets[qc] = (long long)hc[3 * qc + 1];
            if (!timed[qc]) stats->class_ms[qc] = 0.0;
            q += (long long)hc[3 * qc];
            pq += (long long)hc[3 * qc + 1];
            q32 += (long long)hc[3 * qc + 2];
        }
        stats->quartets = q;
        stats->prim_quartets = pq;
        stats->fp32_quartets = q32;
        stats->pairs = npairs_kept;
        stats->tiles = (long long)tiles_all.size();
        stats->launches = launches;
        stats->grid = G;
        stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    return TG_OK;
}

}  // extern "C"
