// C-ABI of libtdgrad and the host-side planner: basis upload, Schwarz
// factors, pair screening and class sort, quartet tiles, class launches and
// the final reduction.  Every arithmetic step of the gradient runs in the
// CUDA kernels; the host only orders work and moves buffers.
#include <algorithm>
#include <cstdio>
#include <cstdint>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <new>
#include <vector>

#include "class_launchers.cuh"
#include "plan_kernels.cuh"
#include "router.cuh"
#include "setup_kernels.cuh"

using namespace tg;

namespace {

// Test hook for the allocation-failure path: while the environment variable
// TDGRAD_FAIL_ALLOC is set to 1, every arena growth fails as if cudaMalloc had
// run out of device memory (checked on the host; no CUDA call is made).
bool alloc_failure_injected()
{
    const char *e = std::getenv("TDGRAD_FAIL_ALLOC");
    return e && e[0] == '1' && e[1] == 0;
}

struct DevArena {
    char *p = nullptr;
    size_t cap = 0;
    size_t used = 0;
    cudaError_t reserve(size_t bytes)
    {
        if (bytes <= cap) return cudaSuccess;
        if (alloc_failure_injected()) return cudaErrorMemoryAllocation;
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

struct tg_router {
    float params[NPARAM];
    float mu[NFEAT], sd[NFEAT];
    float margin = 0.f;   // added to predictions (log10) before routing
    float eps_rel = 0.f;  // fp32 error of a quartet relative to its largest contribution
    int trained = 0;
};

struct tg_basis {
    int device = 0;
    int natom = 0, nshell = 0, nbf = 0, nprim = 0;
    std::vector<int> sh_atom, sh_l, sh_nprim, sh_poff, sh_bf;
    double *d_xyz = nullptr, *d_exps = nullptr, *d_coefs = nullptr, *d_cn = nullptr, *d_boys = nullptr;
    int *d_sh_atom = nullptr, *d_sh_l = nullptr, *d_sh_nprim = nullptr, *d_sh_poff = nullptr, *d_sh_bf = nullptr;
    std::vector<double> Q, Qd;  // per canonical pair key (x >= y)
    double Qmax = 0.0, Qdmax = 0.0;
    long long *d_bpoff = nullptr;  // per canonical pair key: offset of its primitive-pair bounds
    double *d_bp = nullptr;        // primitive-pair bounds b_kl (larger shell index first)
    DevArena ws1, ws2;
    DevArena ws3, ws4;  // device tile planner: per-class tile maxima and rows; tile lists
    DevArena ws5;       // Fock build: densities, combined matrices, F
    float *d_router = nullptr;  // router parameters, mean and std on the device
    int nsm = 0;
    // tg_grad2e's autotuner (tg_options.autotune = 1): kernel form, grid cap
    // and bra-primitive splits per (class, precision) list, chosen on the
    // first such call and kept for the later ones
    bool tuned = false;
    int tune_kind[2 * NQC], tune_grid[2 * NQC], tune_split[2 * NQC];
    // spherical shells: 2l+1 functions per shell; per Cartesian function its
    // shell's first spherical function << 8 | l << 4 | Cartesian component
    int nsph = 0;
    std::vector<int> cmap;
    DevArena ws6;  // tg_grad2e_sph: spherical and Cartesian densities, gradient
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
    cudaFree(b->d_router);
    cudaFree(b->d_bpoff);
    cudaFree(b->d_bp);
    b->ws1.release();
    b->ws2.release();
    b->ws3.release();
    b->ws4.release();
    b->ws5.release();
    b->ws6.release();
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
    TG_CUDA(cudaMalloc(&b->d_boys, (sizeof(double) + sizeof(float)) * BOYS_TAB));
    TG_CUDA(cudaMalloc(&b->d_router, sizeof(float) * (NPARAM + 2 * NFEAT)));
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
    std::vector<long long> bpoff((size_t)npr + 1);
    {
        long long o = 0;
        for (long long k = 0; k < npr; ++k) {
            bpoff[(size_t)k] = o;
            o += (long long)b->sh_nprim[prs[(size_t)k].x] * b->sh_nprim[prs[(size_t)k].y];
        }
        bpoff[(size_t)npr] = o;
    }
    int2 *d_prs = nullptr;
    double *d_Q = nullptr, *d_Qd = nullptr;
    cudaError_t e = cudaMalloc(&d_prs, sizeof(int2) * npr);
    if (e == cudaSuccess) e = cudaMalloc(&d_Q, sizeof(double) * npr);
    if (e == cudaSuccess) e = cudaMalloc(&d_Qd, sizeof(double) * npr);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_bpoff, sizeof(long long) * (npr + 1));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_bp, sizeof(double) * std::max<long long>(bpoff[(size_t)npr], 1));
    if (e == cudaSuccess) e = cudaMemcpy(d_prs, prs.data(), sizeof(int2) * npr, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(b->d_bpoff, bpoff.data(), sizeof(long long) * (npr + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        k_schwarz<<<(unsigned)((npr + 127) / 128), 128>>>((int)npr, d_prs, b->d_xyz, b->d_sh_atom, b->d_sh_l,
                                                          b->d_sh_nprim, b->d_sh_poff, b->d_exps, b->d_cn, d_Q, d_Qd,
                                                          b->d_bpoff, b->d_bp);
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

// fp32 relative error assumed by the bound router, per quartet, relative to
// nfq * bound (see tg_grad2e)
constexpr double kEps32Bound = 3e-6;

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
    o->autotune = 0;
    o->kernel_kind = TG_KERNEL_DEFAULT;
    o->deterministic = 1;
    o->class_mask = 0;
}

int tg_abi_version(void) { return TG_ABI_VERSION; }

int tg_tile_shard(long long ntiles, int rank, int nranks, long long *first, long long *count, long long *stride)
{
    if (ntiles < 0 || nranks < 1 || rank < 0 || rank >= nranks || !first || !count || !stride) return TG_EINVAL;
    *first = rank;
    *stride = nranks;
    *count = ntiles > rank ? (ntiles - rank + nranks - 1) / nranks : 0;
    return TG_OK;
}

const char *tg_strerror(int s)
{
    switch (s) {
    case TG_OK: return "ok";
    case TG_EINVAL: return "invalid argument";
    case TG_EUNSUPPORTED: return "unsupported input (l > 2, several lr omegas, too many pairs, size beyond int32 indexing)";
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
    int po = 0, bo = 0, so = 0;
    b->cmap.resize(nbf);
    for (int s = 0; s < nshell; ++s) {
        b->sh_poff[s] = po;
        b->sh_bf[s] = bo;
        for (int c = 0; c < ncart(shell_l[s]); ++c) b->cmap[bo + c] = (so << 8) | (shell_l[s] << 4) | c;
        po += shell_nprim[s];
        bo += ncart(shell_l[s]);
        so += 2 * shell_l[s] + 1;
    }
    b->nsph = so;
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
int tg_basis_nsph(const tg_basis *b) { return b ? b->nsph : TG_EINVAL; }

void tg_basis_destroy(tg_basis *b)
{
    if (!b) return;
    free_basis(b);
    delete b;
}

}  // extern "C"

namespace {

struct HostTile {
    unsigned bt, kt;
    long long cost;
    double bnd;  // rigorous bound of any per-function-quartet contribution in the tile
    int qc;
};

// Host plan of one call: device densities and block factors, screened and
// sorted shell pairs, primitive-pair records, and the unrouted tile list.
struct Plan {
    int npair = 0;
    DensArgs den;
    GeoArgs geo;
    ScreenArgs scr;
    PrimPairs pp;
    double tau = 0.0, scale = 0.0;
    double *dM = nullptr, *dMrow = nullptr, *dgrad = nullptr;
    unsigned long long *dcnt = nullptr;
    std::vector<double> Mrow;
    std::vector<HostPair> cls[NPC];
    int cls_off[NPC + 1];
    long long npairs_kept = 0, nprimpairs = 0;
    int *d_sa = nullptr, *d_sb = nullptr, *d_poff = nullptr, *d_np = nullptr, *d_key = nullptr;
    double *d_Q = nullptr, *d_Qd = nullptr;
    std::vector<HostTile> tiles;
    int qc_P[NQC], qc_Q[NQC];
    unsigned class_mask = 0;
    bool fock = false;  // Fock build: linear bounds, Q only
    int launches = 0;
    int G = 1;
    PairSet set(int c) const
    {
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
    }
};

int check_pairs(int npair, const tg_pair *pairs, const tg_options &opt, double &omega, int &use_lr)
{
    if (npair < 1 || !pairs) return TG_EINVAL;
    if (npair > TG_MAX_PAIRS) return TG_EUNSUPPORTED;
    if (!(opt.screen_tol >= 0.0) || !std::isfinite(opt.screen_tol)) return TG_EINVAL;
    if (opt.nranks < 1 || opt.rank < 0 || opt.rank >= opt.nranks) return TG_EINVAL;
    if (opt.precision != TG_FP64 && opt.precision != TG_MIXED_BOUND && opt.precision != TG_MIXED_LEARNED &&
        opt.precision != TG_FP32)
        return TG_EINVAL;
    if (!(opt.mixed_tol >= 0.0) || !std::isfinite(opt.mixed_tol)) return TG_EINVAL;
    if (opt.kernel_kind < TG_KERNEL_DEFAULT || opt.kernel_kind > TG_KERNEL_WARP) return TG_EINVAL;
    if (opt.deterministic != 0 && opt.deterministic != 1) return TG_EINVAL;
    if (opt.class_mask >> NQC) return TG_EINVAL;
    for (int r : opt.reserved)
        if (r != 0) return TG_EINVAL;
    if (opt.shard_mode != TG_SHARD_PAIR_KEY && opt.shard_mode != TG_SHARD_TILES) return TG_EINVAL;
    if (opt.autotune < 0 || opt.autotune > 2) return TG_EINVAL;
    omega = 0.0;
    use_lr = 0;
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
    return TG_OK;
}

// Densities, block factors, screened pairs, primitive pairs, unrouted tiles.
int make_plan(tg_basis *b, int npair, const tg_pair *pairs, const tg_options &opt, cudaStream_t st, Plan &pl,
              bool host_tiles = true, bool fock = false)
{
    double omega;
    int use_lr;
    int rc = check_pairs(npair, pairs, opt, omega, use_lr);
    if (rc != TG_OK) return rc;
    const int nbf = b->nbf, ns = b->nshell, natom = b->natom;
    const size_t nbf2 = (size_t)nbf * nbf;
    TG_CUDA(cudaSetDevice(b->device));
    pl.npair = npair;
    std::memset(&pl.den, 0, sizeof(pl.den));
    DensArgs &den = pl.den;
    den.npair = npair;
    den.nbf = nbf;
    den.use_lr = use_lr;
    den.omega = omega;
    for (int p = 0; p < npair; ++p) {
        den.cJ[p] = pairs[p].c_J;
        den.cK[p] = pairs[p].c_K;
        den.cKlr[p] = (pairs[p].omega > 0.0) ? pairs[p].c_K_lr : 0.0;
    }
    // ---- arena 1: densities, symmetrised copies, block factors, output
    DevArena &W = b->ws1;
    const int nmat_up = opt.device_ptrs ? 0 : 2 * npair;
    const size_t need1 = al(sizeof(double) * nbf2) * (nmat_up + 2 * npair) + al(sizeof(double) * (size_t)ns * ns) +
                         al(sizeof(double) * ns) + al(sizeof(double) * TG_MAX_PAIRS) +
                         al(sizeof(double) * 3 * natom) + al(sizeof(unsigned long long) * NCNT * NQC) + 4096;
    TG_CUDA(W.reserve(need1));
    W.used = 0;
    double *dmat[2 * TG_MAX_PAIRS], *dS[2 * TG_MAX_PAIRS];
    for (int k = 0; k < nmat_up; ++k) dmat[k] = W.take<double>(nbf2);
    for (int k = 0; k < 2 * npair; ++k) dS[k] = W.take<double>(nbf2);
    pl.dM = W.take<double>((size_t)ns * ns);
    pl.dMrow = W.take<double>(ns);
    double *dw = W.take<double>(TG_MAX_PAIRS);
    pl.dgrad = W.take<double>(3 * natom);
    pl.dcnt = W.take<unsigned long long>(NCNT * NQC);
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
        pl.launches += 2;
    }
    double hw[TG_MAX_PAIRS];
    for (int p = 0; p < npair; ++p)
        hw[p] = std::sqrt(std::fabs(den.cJ[p]) + std::fabs(den.cK[p]) + std::fabs(den.cKlr[p]));
    TG_CUDA(cudaMemcpyAsync(dw, hw, sizeof(double) * npair, cudaMemcpyHostToDevice, st));
    const long long npr_all = (long long)ns * (ns + 1) / 2;
    k_blockmax<<<(unsigned)((npr_all + 127) / 128), 128, 0, st>>>(ns, b->d_sh_bf, b->d_sh_l, den, dw, pl.dM,
                                                                   pl.dMrow);
    k_rowmax<<<(ns + 127) / 128, 128, 0, st>>>(ns, pl.dM, pl.dMrow);
    pl.launches += 2;
    TG_CUDA(cudaGetLastError());
    pl.Mrow.resize(ns);
    TG_CUDA(cudaMemcpyAsync(pl.Mrow.data(), pl.dMrow, sizeof(double) * ns, cudaMemcpyDeviceToHost, st));
    TG_CUDA(cudaStreamSynchronize(st));
    double Mmax = 0.0;
    for (int x = 0; x < ns; ++x) Mmax = std::max(Mmax, pl.Mrow[x]);

    // ---- pair screening and class sort (Sec. II.C: presort by K and the Schwarz bound)
    pl.tau = opt.screen_tol;
    // gradient: 8 npair max(Q' Q, Q Q') M^2; Fock build: 8 Q Q M (see tdgrad.h)
    pl.fock = fock;
    pl.scale = fock ? 8.0 : 8.0 * npair;
    const double tau = pl.tau, scale = pl.scale;
    for (int x = 0; x < ns; ++x)
        for (int y = 0; y <= x; ++y) {
            const long long k = pkey(x, y);
            const double q = b->Q[(size_t)k], qd = b->Qd[(size_t)k];
            if (tau > 0.0) {
                const double bnd = fock ? scale * q * b->Qmax * Mmax
                                        : scale * std::max(qd * b->Qmax, q * b->Qdmax) * Mmax * Mmax;
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
            pl.cls[pair_class(b->sh_l[sa], b->sh_l[sb])].push_back(hp);
        }
    // surviving primitive pairs per kept shell pair (primitive screen, see tdgrad.h)
    // (the kernels test scale * b_kl * qq * m^2 < eps_p; the Fock build's linear
    // bound scale * b_kl * Qmax * Mmax takes m = sqrt(Mmax))
    const double eps_p = tau > 0.0 ? 1e-6 * tau : 0.0;
    const double qq = fock ? b->Qmax : std::max(b->Qmax, b->Qdmax);
    const double Mp = fock ? std::sqrt(Mmax) : Mmax;
    long long nk_all = 0, npp_max = 0;
    for (int c = 0; c < NPC; ++c) {
        nk_all += (long long)pl.cls[c].size();
        for (auto &hp : pl.cls[c]) npp_max += hp.np;
    }
    // primitive-pair offsets are int32 on the device
    if (npp_max > 0x7fffffffLL) return TG_EUNSUPPORTED;
    // ---- arena 2: pair arrays, primitive-pair records, tiles, features, partials
    pl.G = std::max(1, 4 * b->nsm);  // partial slabs: up to 4 resident CTAs per SM
    {
        const size_t np_k = (size_t)std::max<long long>(nk_all, 1);
        const size_t npp = (size_t)std::max<long long>(npp_max, 1);
        // tiles: at most one per (bra tile, ket tile) combination of every class
        long long ntl_max = 0;
        for (int P = 0; P < NPC; ++P)
            for (int Qc = 0; Qc <= P; ++Qc)
                ntl_max += (long long)((pl.cls[P].size() + TB - 1) / TB) * ((pl.cls[Qc].size() + TK - 1) / TK);
        const size_t ntl = host_tiles ? (size_t)std::max<long long>(ntl_max, 1) : 1;
        const size_t need2 = 6 * al(sizeof(int) * np_k) + 2 * al(sizeof(double) * np_k) +
                             6 * al(sizeof(double) * npp) + 12 * al(sizeof(float) * npp) + al(sizeof(uint4) * ntl) +
                             al(sizeof(MolDesc)) +
                             al(sizeof(TileRef) * ntl) + al(sizeof(float) * ntl * (NFEAT + 1)) +
                             al(sizeof(double) * (size_t)pl.G * 3 * natom) + 8192;
        DevArena &V = b->ws2;
        TG_CUDA(V.reserve(need2));
        V.used = 0;
        pl.d_sa = V.take<int>(np_k);
        pl.d_sb = V.take<int>(np_k);
        pl.d_poff = V.take<int>(np_k);
        pl.d_np = V.take<int>(np_k);
        pl.d_key = V.take<int>(np_k);
        pl.d_Q = V.take<double>(np_k);
        pl.d_Qd = V.take<double>(np_k);
        int *d_cnt = V.take<int>(np_k);
        std::vector<int> u_sa, u_sb, u_key;
        for (int c = 0; c < NPC; ++c)
            for (auto &hp : pl.cls[c]) {
                u_sa.push_back(hp.sa);
                u_sb.push_back(hp.sb);
                u_key.push_back(hp.key);
            }
        if (nk_all > 0) {
            TG_CUDA(cudaMemcpyAsync(pl.d_sa, u_sa.data(), sizeof(int) * nk_all, cudaMemcpyHostToDevice, st));
            TG_CUDA(cudaMemcpyAsync(pl.d_sb, u_sb.data(), sizeof(int) * nk_all, cudaMemcpyHostToDevice, st));
            TG_CUDA(cudaMemcpyAsync(pl.d_key, u_key.data(), sizeof(int) * nk_all, cudaMemcpyHostToDevice, st));
            k_prim_count<<<(unsigned)((nk_all + 127) / 128), 128, 0, st>>>((int)nk_all, pl.d_sa, pl.d_sb, pl.d_key,
                                                                           b->d_sh_nprim, b->d_bpoff, b->d_bp, scale,
                                                                           qq, Mp, eps_p, d_cnt);
            ++pl.launches;
            TG_CUDA(cudaGetLastError());
            std::vector<int> cnt((size_t)nk_all);
            TG_CUDA(cudaMemcpyAsync(cnt.data(), d_cnt, sizeof(int) * nk_all, cudaMemcpyDeviceToHost, st));
            TG_CUDA(cudaStreamSynchronize(st));
            size_t i = 0;
            for (int c = 0; c < NPC; ++c) {
                std::vector<HostPair> kept;
                for (auto &hp : pl.cls[c]) {
                    hp.np = cnt[i++];
                    if (hp.np > 0) kept.push_back(hp);
                }
                pl.cls[c].swap(kept);
            }
        }
    }
    std::vector<int> h_sa, h_sb, h_poff, h_np, h_key;
    std::vector<double> h_Q, h_Qd;
    {
        int po = 0, n = 0;
        for (int c = 0; c < NPC; ++c) {
            std::sort(pl.cls[c].begin(), pl.cls[c].end(), [](const HostPair &u, const HostPair &v) {
                if (u.np != v.np) return u.np > v.np;
                if (u.Qd != v.Qd) return u.Qd > v.Qd;
                return u.key < v.key;
            });
            pl.cls_off[c] = n;
            for (auto &hp : pl.cls[c]) {
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
        pl.cls_off[NPC] = n;
        pl.npairs_kept = n;
        pl.nprimpairs = po;
    }

    // ---- unrouted quartet tiles with their bounds (screened); the device
    // planner (device_tiles) builds the same list on the GPU instead
    for (int P = 0; P < NPC; ++P)
        for (int Qc = 0; Qc <= P; ++Qc) {
            pl.qc_P[P * (P + 1) / 2 + Qc] = P;
            pl.qc_Q[P * (P + 1) / 2 + Qc] = Qc;
        }
    pl.class_mask = opt.class_mask;
    auto blockmax = [&](int c, int blk, int bsz, double &q, double &qd, double &m) {
        q = qd = m = 0.0;
        const int lo = blk * bsz, hi = std::min((int)pl.cls[c].size(), lo + bsz);
        for (int i = lo; i < hi; ++i) {
            const HostPair &hp = pl.cls[c][i];
            q = std::max(q, hp.Q);
            qd = std::max(qd, hp.Qd);
            m = std::max(m, std::max(pl.Mrow[hp.sa], pl.Mrow[hp.sb]));
        }
    };
    for (int qc = 0; qc < NQC && host_tiles; ++qc) {
        if (opt.class_mask && !((opt.class_mask >> qc) & 1u)) continue;
        const int P = pl.qc_P[qc], Qc = pl.qc_Q[qc];
        const int nP = (int)pl.cls[P].size(), nQ = (int)pl.cls[Qc].size();
        if (!nP || !nQ) continue;
        const int nbt = (nP + TB - 1) / TB, nkt = (nQ + TK - 1) / TK;
        std::vector<double> bq(nbt), bqd(nbt), bm(nbt), kq(nkt), kqd(nkt), km(nkt);
        for (int i = 0; i < nbt; ++i) blockmax(P, i, TB, bq[i], bqd[i], bm[i]);
        for (int i = 0; i < nkt; ++i) blockmax(Qc, i, TK, kq[i], kqd[i], km[i]);
        for (int bt = 0; bt < nbt; ++bt)
            for (int kt = 0; kt < nkt; ++kt) {
                if (P == Qc && kt * TK > bt * TB + TB - 1) continue;
                const double Mt = std::max(bm[bt], km[kt]);
                const double bnd = scale * std::max(bqd[bt] * kq[kt], bq[bt] * kqd[kt]) * Mt * Mt;
                if (tau > 0.0 && bnd < tau) continue;
                HostTile t;
                t.bt = bt;
                t.kt = kt;
                t.cost = (long long)pl.cls[P][bt * TB].np * pl.cls[Qc][kt * TK].np;
                t.bnd = bnd;
                t.qc = qc;
                pl.tiles.push_back(t);
            }
    }

    DevArena &V = b->ws2;
    const size_t npp = (size_t)std::max<long long>(pl.nprimpairs, 1);
    double *pp_p = V.take<double>(npp), *pp_x = V.take<double>(npp), *pp_y = V.take<double>(npp),
           *pp_z = V.take<double>(npp), *pp_K = V.take<double>(npp), *pp_za = V.take<double>(npp);
    float *fp_p = V.take<float>(npp), *fp_x = V.take<float>(npp), *fp_y = V.take<float>(npp),
          *fp_z = V.take<float>(npp), *fp_K = V.take<float>(npp), *fp_za = V.take<float>(npp);
    float *fp_PA = V.take<float>(3 * npp), *fp_PB = V.take<float>(3 * npp);
    const long long nk = pl.npairs_kept;
    if (nk > 0) {
        TG_CUDA(cudaMemcpyAsync(pl.d_sa, h_sa.data(), sizeof(int) * nk, cudaMemcpyHostToDevice, st));
        TG_CUDA(cudaMemcpyAsync(pl.d_sb, h_sb.data(), sizeof(int) * nk, cudaMemcpyHostToDevice, st));
        TG_CUDA(cudaMemcpyAsync(pl.d_poff, h_poff.data(), sizeof(int) * nk, cudaMemcpyHostToDevice, st));
        TG_CUDA(cudaMemcpyAsync(pl.d_np, h_np.data(), sizeof(int) * nk, cudaMemcpyHostToDevice, st));
        TG_CUDA(cudaMemcpyAsync(pl.d_key, h_key.data(), sizeof(int) * nk, cudaMemcpyHostToDevice, st));
        TG_CUDA(cudaMemcpyAsync(pl.d_Q, h_Q.data(), sizeof(double) * nk, cudaMemcpyHostToDevice, st));
        TG_CUDA(cudaMemcpyAsync(pl.d_Qd, h_Qd.data(), sizeof(double) * nk, cudaMemcpyHostToDevice, st));
        k_prim_pairs<<<(unsigned)((nk + 127) / 128), 128, 0, st>>>(
            (int)nk, pl.d_sa, pl.d_sb, pl.d_poff, pl.d_key, b->d_xyz, b->d_sh_atom, b->d_sh_nprim, b->d_sh_poff,
            b->d_exps, b->d_cn, b->d_bpoff, b->d_bp, scale, qq, Mp, eps_p, pp_p, pp_x, pp_y, pp_z, pp_K, pp_za, fp_p,
            fp_x, fp_y, fp_z, fp_K, fp_za, fp_PA, fp_PB, (long long)npp);
        ++pl.launches;
        TG_CUDA(cudaGetLastError());
        // the host pair vectors must outlive the asynchronous copies
        TG_CUDA(cudaStreamSynchronize(st));
    }
    pl.pp.p = pp_p;
    pl.pp.Px = pp_x;
    pl.pp.Py = pp_y;
    pl.pp.Pz = pp_z;
    pl.pp.K = pp_K;
    pl.pp.za = pp_za;
    pl.pp.fp = fp_p;
    pl.pp.fPx = fp_x;
    pl.pp.fPy = fp_y;
    pl.pp.fPz = fp_z;
    pl.pp.fK = fp_K;
    pl.pp.fza = fp_za;
    pl.pp.fPA = fp_PA;
    pl.pp.fPB = fp_PB;
    pl.pp.n = (long long)npp;
    pl.geo.natom = natom;
    pl.geo.nshell = ns;
    pl.geo.xyz = b->d_xyz;
    pl.geo.sh_atom = b->d_sh_atom;
    pl.geo.sh_bf = b->d_sh_bf;
    pl.scr.tau = tau;
    pl.scr.scale = scale;
    pl.scr.M = pl.dM;
    pl.scr.nshell = ns;
    // the pair-key shard filter runs inside the class kernels; tile shards select tiles
    pl.scr.rank = opt.shard_mode == TG_SHARD_TILES ? 0 : opt.rank;
    pl.scr.nranks = opt.shard_mode == TG_SHARD_TILES ? 1 : opt.nranks;
    return TG_OK;
}

FeatureArgs feature_args(const tg_basis *b, const Plan &pl)
{
    FeatureArgs fa;
    for (int c = 0; c < NPC; ++c) fa.sets[c] = pl.set(c);
    fa.M = pl.dM;
    fa.xyz = b->d_xyz;
    fa.sh_atom = b->d_sh_atom;
    fa.pp_p = pl.pp.p;
    fa.nshell = b->nshell;
    fa.scale = pl.scale;
    return fa;
}

// Features and router predictions (log10 magnitude) for the listed tiles.
int predict_tiles(tg_basis *b, const Plan &pl, const tg_router *r, const std::vector<size_t> &idx, cudaStream_t st,
                  TileRef *d_ref, float *d_feat, float *d_pred, std::vector<float> *pred, std::vector<float> *feat,
                  int &launches)
{
    const size_t n = idx.size();
    if (!n) return TG_OK;
    std::vector<TileRef> refs(n);
    for (size_t i = 0; i < n; ++i) {
        const HostTile &t = pl.tiles[idx[i]];
        refs[i].P = pl.qc_P[t.qc];
        refs[i].Q = pl.qc_Q[t.qc];
        refs[i].bt = t.bt;
        refs[i].kt = t.kt;
    }
    TG_CUDA(cudaMemcpyAsync(d_ref, refs.data(), sizeof(TileRef) * n, cudaMemcpyHostToDevice, st));
    k_tile_features<<<(unsigned)((n + 127) / 128), 128, 0, st>>>((int)n, d_ref, feature_args(b, pl), d_feat);
    ++launches;
    TG_CUDA(cudaGetLastError());
    if (r) {
        float *dparams = b->d_router;
        TG_CUDA(cudaMemcpyAsync(dparams, r->params, sizeof(float) * NPARAM, cudaMemcpyHostToDevice, st));
        TG_CUDA(cudaMemcpyAsync(dparams + NPARAM, r->mu, sizeof(float) * NFEAT, cudaMemcpyHostToDevice, st));
        TG_CUDA(cudaMemcpyAsync(dparams + NPARAM + NFEAT, r->sd, sizeof(float) * NFEAT, cudaMemcpyHostToDevice, st));
        k_mlp_predict<<<(unsigned)((n + 127) / 128), 128, 0, st>>>((int)n, d_feat, dparams + NPARAM,
                                                                    dparams + NPARAM + NFEAT, dparams, d_pred);
        ++launches;
        TG_CUDA(cudaGetLastError());
        if (pred) {
            pred->resize(n);
            TG_CUDA(cudaMemcpyAsync(pred->data(), d_pred, sizeof(float) * n, cudaMemcpyDeviceToHost, st));
        }
    }
    if (feat) {
        feat->resize(n * NFEAT);
        TG_CUDA(cudaMemcpyAsync(feat->data(), d_feat, sizeof(float) * n * NFEAT, cudaMemcpyDeviceToHost, st));
    }
    TG_CUDA(cudaStreamSynchronize(st));
    return TG_OK;
}

// Routing of one molecule's tiles.  e_t estimates tile t's fp32 error in any
// single gradient component: eps * (every gradient component of a quartet is
// at most nfq * bound, and a tile holds TILE quartets) for the bound router,
// eps_rel * 10^(prediction + margin) for the learned router, whose prediction
// is the tile's largest contribution to one gradient component.  Tiles go to
// fp32 in increasing e_t while sum e_t^2 stays within mixed_tol^2: the fp32
// rounding errors of different tiles are independent, so they add in
// quadrature.  The safety margin lives in the estimates themselves (the
// bound router's rigorous bound; the learned router's margin, calibrated on
// measured errors against fp64).
int compute_route(tg_basis *b, const Plan &pl, const tg_options &opt, cudaStream_t st, TileRef *d_ref, float *d_feat,
                  float *d_pred, std::vector<uint8_t> &route, int &launches)
{
    const size_t ntl = pl.tiles.size();
    route.assign(ntl, 0);
    if (opt.precision == TG_FP32) {
        std::fill(route.begin(), route.end(), 1);
    } else if (opt.precision == TG_MIXED_BOUND || opt.precision == TG_MIXED_LEARNED) {
        std::vector<double> err(ntl);
        if (opt.precision == TG_MIXED_BOUND) {
            for (size_t i = 0; i < ntl; ++i) {
                const int P = pl.qc_P[pl.tiles[i].qc], Qc = pl.qc_Q[pl.tiles[i].qc];
                const int nfq = ncart(pc_la(P)) * ncart(pc_lb(P)) * ncart(pc_la(Qc)) * ncart(pc_lb(Qc));
                err[i] = kEps32Bound * TILE * nfq * pl.tiles[i].bnd;
            }
        } else {
            std::vector<size_t> all(ntl);
            for (size_t i = 0; i < ntl; ++i) all[i] = i;
            std::vector<float> pred;
            int rc = predict_tiles(b, pl, opt.router, all, st, d_ref, d_feat, d_pred, &pred, nullptr, launches);
            if (rc != TG_OK) return rc;
            for (size_t i = 0; i < ntl; ++i)
                err[i] = (double)opt.router->eps_rel * std::pow(10.0, (double)pred[i] + opt.router->margin);
        }
        std::vector<size_t> ord(ntl);
        for (size_t i = 0; i < ntl; ++i) ord[i] = i;
        std::stable_sort(ord.begin(), ord.end(), [&](size_t u, size_t v) { return err[u] < err[v]; });
        const double budget = opt.mixed_tol * opt.mixed_tol;
        double acc = 0.0;
        for (size_t i : ord) {
            if (acc + err[i] * err[i] > budget) break;
            acc += err[i] * err[i];
            route[i] = 1;
        }
    }
    return TG_OK;
}

// Tile lists of one call built on the device (row a3 of the hot path): tile
// maxima per class, the hierarchical block screen (plan_kernels.cu) counting
// and then writing the kept tiles of every (class, bra tile) row, fp32 /
// fp64 routing from a histogram of the tiles' error estimates, and an
// order-preserving split into the (class, precision) launch lists.  The host
// only prefix-sums per-row counts and picks the routing cut-off from the
// histogram.  Routing: tiles go to fp32 bin by bin in increasing error while
// the sum of e_t^2, each e_t taken at its bin's upper edge, stays within
// mixed_tol^2 -- the rule of compute_route, with bins of 2^(1/8).
struct DevTiles {
    uint4 *tiles = nullptr;  // launch lists, [class][fp64 | fp32]
    long long off[2 * NQC + 1];
    long long ntiles = 0;
    int cut = 0;
};

int device_tiles(tg_basis *b, const Plan &pl, const tg_options &opt, cudaStream_t st, DevTiles &dt, int &launches)
{
    // rows (class, bra tile, ket tile run): the ket tiles of a class split into
    // runs of equal cost factor (primitive pairs of a tile's first pair; the
    // pairs are sorted by it), every row of a class has one cost, and the rows
    // of a class are sorted stably by decreasing cost -- the tile order of the
    // host planner (build_exec)
    std::vector<int4> rows;
    int row_qc_begin[NQC + 1];
    {
        std::vector<std::vector<int2>> runs(NPC);  // (first ket tile, end) per pair class
        for (int c = 0; c < NPC; ++c) {
            const int n = (int)pl.cls[c].size(), nk = (n + TK - 1) / TK;
            for (int kt = 0; kt < nk;) {
                int e = kt + 1;
                while (e < nk && pl.cls[c][e * TK].np == pl.cls[c][kt * TK].np) ++e;
                runs[c].push_back(make_int2(kt, e));
                kt = e;
            }
        }
        std::vector<std::pair<long long, int4>> tmp;
        for (int qc = 0; qc < NQC; ++qc) {
            row_qc_begin[qc] = (int)rows.size();
            if (pl.class_mask && !((pl.class_mask >> qc) & 1u)) continue;
            const int P = pl.qc_P[qc], Qc = pl.qc_Q[qc];
            const int nP = (int)pl.cls[P].size(), nQ = (int)pl.cls[Qc].size();
            if (!nP || !nQ) continue;
            tmp.clear();
            for (int bt = 0; bt < (nP + TB - 1) / TB; ++bt) {
                const long long cb = pl.cls[P][bt * TB].np;
                const int lim = P == Qc ? (bt * TB + TB - 1) / TK + 1 : (nQ + TK - 1) / TK;  // canonical limit
                for (const int2 &ru : runs[Qc]) {
                    if (ru.x >= lim) break;
                    tmp.push_back({cb * pl.cls[Qc][ru.x * TK].np, make_int4(qc, bt, ru.x, std::min(ru.y, lim))});
                }
            }
            std::stable_sort(tmp.begin(), tmp.end(),
                             [](const std::pair<long long, int4> &u, const std::pair<long long, int4> &v) {
                                 return u.first > v.first;
                             });
            for (auto &t : tmp) rows.push_back(t.second);
        }
        row_qc_begin[NQC] = (int)rows.size();
    }
    const int nrows = (int)rows.size();
    for (int k = 0; k <= 2 * NQC; ++k) dt.off[k] = 0;
    dt.ntiles = 0;
    if (!nrows) return TG_OK;
    // ---- phase A buffers: tile maxima, rows, per-row counts and offsets
    RowArgs ra;
    std::memset(&ra, 0, sizeof(ra));
    ra.nrows = nrows;
    ra.tau = pl.tau;
    ra.scale = pl.scale;
    ra.fock = pl.fock ? 1 : 0;
    for (int qc = 0; qc < NQC; ++qc) {
        ra.qcP[qc] = pl.qc_P[qc];
        ra.qcQ[qc] = pl.qc_Q[qc];
    }
    size_t needA = al(sizeof(int4) * nrows) + 3 * al(sizeof(int) * (nrows + 1)) +
                   4 * al(sizeof(long long) * (nrows + 1)) + al(sizeof(unsigned long long) * RBIN_N) + 4096;
    for (int c = 0; c < NPC; ++c) {
        const size_t n = pl.cls[c].size();
        const size_t nb = (n + TB - 1) / TB, nk = (n + TK - 1) / TK, ng = (nk + GROUP - 1) / GROUP;
        needA += 3 * (al(sizeof(double) * std::max<size_t>(nb, 1)) + al(sizeof(double) * std::max<size_t>(nk, 1)) +
                      al(sizeof(double) * std::max<size_t>(ng, 1)));
    }
    DevArena &A = b->ws3;
    TG_CUDA(A.reserve(needA));
    A.used = 0;
    for (int c = 0; c < NPC; ++c) {
        const int n = (int)pl.cls[c].size();
        const int nb = (n + TB - 1) / TB, nk = (n + TK - 1) / TK, ng = (nk + GROUP - 1) / GROUP;
        TileMaxima &t = ra.t[c];
        double *bq = A.take<double>(std::max(nb, 1)), *bqd = A.take<double>(std::max(nb, 1)),
               *bm = A.take<double>(std::max(nb, 1));
        double *kq = A.take<double>(std::max(nk, 1)), *kqd = A.take<double>(std::max(nk, 1)),
               *km = A.take<double>(std::max(nk, 1));
        double *gq = A.take<double>(std::max(ng, 1)), *gqd = A.take<double>(std::max(ng, 1)),
               *gm = A.take<double>(std::max(ng, 1));
        t.bq = bq; t.bqd = bqd; t.bm = bm; t.kq = kq; t.kqd = kqd; t.km = km; t.gq = gq; t.gqd = gqd; t.gm = gm;
        t.nbt = nb;
        t.nkt = nk;
        if (!n) continue;
        const PairSet ps = pl.set(c);
        k_tile_maxima<<<(nb + 127) / 128, 128, 0, st>>>(n, TB, ps.sa, ps.sb, ps.Q, ps.Qd, pl.dMrow, bq, bqd, bm);
        k_tile_maxima<<<(nk + 127) / 128, 128, 0, st>>>(n, TK, ps.sa, ps.sb, ps.Q, ps.Qd, pl.dMrow, kq, kqd, km);
        k_group_maxima<<<(ng + 127) / 128, 128, 0, st>>>(nk, kq, kqd, km, gq, gqd, gm);
        launches += 3;
    }
    int4 *d_rows = A.take<int4>(nrows);
    int *d_cnt = A.take<int>(nrows + 1), *d_cnt32 = A.take<int>(nrows + 1), *d_cntk = A.take<int>(nrows + 1);
    long long *d_off = A.take<long long>(nrows + 1), *d_o64 = A.take<long long>(nrows + 1),
              *d_o32 = A.take<long long>(nrows + 1), *d_base = A.take<long long>(nrows + 1);
    unsigned long long *d_hist = A.take<unsigned long long>(RBIN_N);
    ra.rows = d_rows;
    TG_CUDA(cudaMemcpyAsync(d_rows, rows.data(), sizeof(int4) * nrows, cudaMemcpyHostToDevice, st));
    const unsigned gr = (unsigned)((nrows + 127) / 128);
    k_tile_rows<<<gr, 128, 0, st>>>(ra, 0, d_cnt, nullptr, nullptr, nullptr);
    ++launches;
    TG_CUDA(cudaGetLastError());
    std::vector<int> cnt(nrows);
    TG_CUDA(cudaMemcpyAsync(cnt.data(), d_cnt, sizeof(int) * nrows, cudaMemcpyDeviceToHost, st));
    TG_CUDA(cudaStreamSynchronize(st));
    std::vector<long long> off(nrows + 1);
    off[0] = 0;
    for (int r = 0; r < nrows; ++r) off[r + 1] = off[r] + cnt[r];
    const long long ntl = off[nrows];
    dt.ntiles = ntl;
    if (!ntl) return TG_OK;
    // start of each row's class in the screened list (the tile shard deals
    // every class list round-robin from there)
    std::vector<long long> base(nrows + 1, 0);
    for (int qc = 0; qc < NQC; ++qc)
        for (int r = row_qc_begin[qc]; r < row_qc_begin[qc + 1]; ++r) base[r] = off[row_qc_begin[qc]];
    const bool tshard = opt.shard_mode == TG_SHARD_TILES && opt.nranks > 1;
    const int srank = tshard ? opt.rank : 0, snr = tshard ? opt.nranks : 1;
    TG_CUDA(cudaMemcpyAsync(d_off, off.data(), sizeof(long long) * (nrows + 1), cudaMemcpyHostToDevice, st));
    TG_CUDA(cudaMemcpyAsync(d_base, base.data(), sizeof(long long) * (nrows + 1), cudaMemcpyHostToDevice, st));
    // ---- phase B buffers: the tiles, their bounds and routing bins (24 B per
    // screened tile), this rank's launch lists (16 B per tile of the shard) and,
    // for the learned router, feature and prediction buffers for one chunk of
    // at most RCHUNK tiles at a time
    const bool learned = opt.precision == TG_MIXED_LEARNED, bound = opt.precision == TG_MIXED_BOUND;
    constexpr long long RCHUNK = 1LL << 25;
    const long long nout = snr > 1 ? std::min(ntl, ntl / snr + 2 * NQC) : ntl;  // a class list of n deals <= n/snr + 1
    const long long nch = std::min(ntl, RCHUNK);
    size_t needB = al(sizeof(uint4) * ntl) + al(sizeof(uint4) * nout) + al(sizeof(float) * ntl) +
                   al(sizeof(int) * ntl) + 4096;
    if (learned) needB += al(sizeof(TileRef) * nch) + al(sizeof(float) * nch * NFEAT) + al(sizeof(float) * nch);
    DevArena &B = b->ws4;
    TG_CUDA(B.reserve(needB));
    B.used = 0;
    uint4 *d_raw = B.take<uint4>(ntl), *d_out = B.take<uint4>(nout);
    float *d_bnd = B.take<float>(ntl);
    int *d_bin = B.take<int>(ntl);
    k_tile_rows<<<gr, 128, 0, st>>>(ra, 1, nullptr, d_off, d_raw, d_bnd);
    ++launches;
    TG_CUDA(cudaGetLastError());
    // grid-stride routing-bin launches: a few blocks per SM, each with its own histogram
    const unsigned gbin = (unsigned)std::max<long long>(1, std::min<long long>((ntl + 127) / 128, 8LL * b->nsm));
    const size_t hbytes = sizeof(unsigned int) * RBIN_N;
    int cut = 0;
    const int *bins = nullptr;
    if (opt.precision == TG_FP32) {
        cut = 1;
    } else if (bound || learned) {
        TG_CUDA(cudaMemsetAsync(d_hist, 0, sizeof(unsigned long long) * RBIN_N, st));
        if (bound) {
            k_route_bins<<<gbin, 128, hbytes, st>>>(ntl, d_raw, d_bnd, 0, kEps32Bound * TILE, 0.0, ra, d_bin, d_hist);
            ++launches;
        } else {
            TileRef *d_ref = B.take<TileRef>(nch);
            float *d_feat = B.take<float>(nch * NFEAT), *d_pred = B.take<float>(nch);
            const tg_router *r = opt.router;
            float *dparams = b->d_router;
            TG_CUDA(cudaMemcpyAsync(dparams, r->params, sizeof(float) * NPARAM, cudaMemcpyHostToDevice, st));
            TG_CUDA(cudaMemcpyAsync(dparams + NPARAM, r->mu, sizeof(float) * NFEAT, cudaMemcpyHostToDevice, st));
            TG_CUDA(cudaMemcpyAsync(dparams + NPARAM + NFEAT, r->sd, sizeof(float) * NFEAT, cudaMemcpyHostToDevice,
                                    st));
            for (long long c0 = 0; c0 < ntl; c0 += RCHUNK) {
                const long long n = std::min(RCHUNK, ntl - c0);
                const unsigned g = (unsigned)((n + 127) / 128);
                const unsigned gb = (unsigned)std::min<long long>(g, 8LL * b->nsm);
                k_tile_refs<<<g, 128, 0, st>>>(n, d_raw + c0, ra, d_ref);
                k_tile_features<<<g, 128, 0, st>>>((int)n, d_ref, feature_args(b, pl), d_feat);
                k_mlp_predict<<<g, 128, 0, st>>>((int)n, d_feat, dparams + NPARAM, dparams + NPARAM + NFEAT, dparams,
                                                 d_pred);
                k_route_bins<<<gb, 128, hbytes, st>>>(n, d_raw + c0, d_pred, 1, (double)r->eps_rel,
                                                      (double)r->margin, ra, d_bin + c0, d_hist);
                launches += 4;
            }
        }
        TG_CUDA(cudaGetLastError());
        std::vector<unsigned long long> hist(RBIN_N);
        TG_CUDA(cudaMemcpyAsync(hist.data(), d_hist, sizeof(unsigned long long) * RBIN_N, cudaMemcpyDeviceToHost, st));
        TG_CUDA(cudaStreamSynchronize(st));
        const double budget = opt.mixed_tol * opt.mixed_tol;
        double acc = 0.0;
        for (int k = 0; k < RBIN_N; ++k) {
            const double u = route_bin_upper(k);
            const double add = (double)hist[k] * u * u;
            if (acc + add > budget) break;
            acc += add;
            cut = k + 1;
        }
        bins = d_bin;
    }
    dt.cut = cut;
    // ---- order-preserving split of this rank's tiles into the (class, precision) lists
    k_row_fp32_count<<<gr, 128, 0, st>>>(nrows, d_off, d_base, srank, snr, bins, cut, d_cnt32, d_cntk);
    ++launches;
    TG_CUDA(cudaGetLastError());
    std::vector<int> c32(nrows), ck(nrows);
    TG_CUDA(cudaMemcpyAsync(c32.data(), d_cnt32, sizeof(int) * nrows, cudaMemcpyDeviceToHost, st));
    TG_CUDA(cudaMemcpyAsync(ck.data(), d_cntk, sizeof(int) * nrows, cudaMemcpyDeviceToHost, st));
    TG_CUDA(cudaStreamSynchronize(st));
    std::vector<long long> o64(nrows), o32(nrows);
    long long pos = 0;
    for (int qc = 0; qc < NQC; ++qc) {
        dt.off[2 * qc] = pos;
        for (int r = row_qc_begin[qc]; r < row_qc_begin[qc + 1]; ++r) {
            o64[r] = pos;
            pos += ck[r] - c32[r];
        }
        dt.off[2 * qc + 1] = pos;
        for (int r = row_qc_begin[qc]; r < row_qc_begin[qc + 1]; ++r) {
            o32[r] = pos;
            pos += c32[r];
        }
    }
    dt.off[2 * NQC] = pos;
    TG_CUDA(cudaMemcpyAsync(d_o64, o64.data(), sizeof(long long) * nrows, cudaMemcpyHostToDevice, st));
    TG_CUDA(cudaMemcpyAsync(d_o32, o32.data(), sizeof(long long) * nrows, cudaMemcpyHostToDevice, st));
    k_row_scatter<<<gr, 128, 0, st>>>(nrows, d_off, d_base, srank, snr, d_raw, bins, cut, d_o64, d_o32, d_out);
    ++launches;
    TG_CUDA(cudaGetLastError());
    // the host vectors must outlive the asynchronous copies
    TG_CUDA(cudaStreamSynchronize(st));
    dt.tiles = d_out;
    return TG_OK;
}

MolDesc make_desc(const Plan &pl, int atom_off)
{
    MolDesc md;
    std::memset(&md, 0, sizeof(md));
    md.geo = pl.geo;
    md.den = pl.den;
    md.scr = pl.scr;
    md.pp = pl.pp;
    for (int c = 0; c < NPC; ++c) md.sets[c] = pl.set(c);
    md.atom_off = atom_off;
    return md;
}

// Two CUDA events for timing, destroyed on every return path.
struct EventPair {
    cudaEvent_t a = nullptr, b = nullptr;
    cudaError_t create()
    {
        cudaError_t e = cudaEventCreate(&a);
        if (e == cudaSuccess) e = cudaEventCreate(&b);
        return e;
    }
    ~EventPair()
    {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
};

// Tiles of a batch per (class, precision), grouped by molecule, each
// molecule's tiles sorted by decreasing cost.
struct Exec {
    std::vector<uint4> tiles;
    long long off[2 * NQC + 1];
    int natom_total = 0, natom_max = 0;
};

void build_exec(const std::vector<const Plan *> &plans, const std::vector<std::vector<uint8_t>> &routes,
                const std::vector<std::vector<size_t>> *subset, Exec &ex)
{
    ex.tiles.clear();
    std::vector<std::vector<std::vector<size_t>>> lists(plans.size(), std::vector<std::vector<size_t>>(2 * NQC));
    for (size_t m = 0; m < plans.size(); ++m) {
        const Plan &pl = *plans[m];
        if (subset) {
            for (size_t i : (*subset)[m]) lists[m][2 * pl.tiles[i].qc + routes[m][i]].push_back(i);
        } else {
            for (size_t i = 0; i < pl.tiles.size(); ++i) lists[m][2 * pl.tiles[i].qc + routes[m][i]].push_back(i);
        }
        if (!subset)
            for (auto &L : lists[m])
                std::stable_sort(L.begin(), L.end(),
                                 [&](size_t u, size_t v) { return pl.tiles[u].cost > pl.tiles[v].cost; });
    }
    for (int k = 0; k < 2 * NQC; ++k) {
        ex.off[k] = (long long)ex.tiles.size();
        for (size_t m = 0; m < plans.size(); ++m)
            for (size_t i : lists[m][k])
                ex.tiles.push_back(make_uint4((unsigned)m, plans[m]->tiles[i].bt, plans[m]->tiles[i].kt, 0u));
    }
    ex.off[2 * NQC] = (long long)ex.tiles.size();
}

// Class launches over an uploaded Exec.  grids[k] (nullable) overrides the
// persistent grid of list k; with dump != nullptr every quartet's 12
// components go to dump[(list position * TILE + thread) * 12 + c].
int launch_exec(const Exec &ex, const MolDesc *d_mols, const uint4 *d_tiles, double *d_part,
                unsigned long long *dcnt, double *dump, const double *boys, int G, const int *grids, bool timing,
                cudaStream_t st, tg_stats *stats, int &launches, const int *kinds = nullptr, int kind_all = 0,
                int tile_rank = 0, int tile_nranks = 1, const int *splits = nullptr)
{
    OutArgs out;
    out.partials = d_part;
    out.natom_total = ex.natom_total;
    out.natom_max = ex.natom_max;
    out.dump = dump;
    const size_t stage = (size_t)TILE * 12 * sizeof(double) + (size_t)TILE * 4 * sizeof(int) +
                         6 * (TB + TK) * sizeof(double) + 2 * (TB + TK) * sizeof(int);
    const size_t sgrad = (size_t)3 * ex.natom_max * sizeof(double);
    out.use_smem = (stage + sgrad) <= 160 * 1024;
    const size_t smem = stage + (out.use_smem ? sgrad : 0);
    EventPair ev;
    if (timing) TG_CUDA(ev.create());
    cudaEvent_t e0 = ev.a, e1 = ev.b;
    int rc = TG_OK;
    for (int qc = 0; qc < NQC && rc == TG_OK; ++qc) {
        for (int r = 0; r < 2; ++r) {
            const int k = 2 * qc + r;
            // tile-cyclic shard: tiles tile_rank, tile_rank + tile_nranks, ... of the list
            long long first = 0, nt = 0, stride = 1;
            tg_tile_shard(ex.off[k + 1] - ex.off[k], tile_rank, tile_nranks, &first, &nt, &stride);
            if (nt <= 0) continue;
            ClassLaunch cl;
            int Pc = 0, Qc = 0;
            for (int a = 0; a < NPC; ++a)
                for (int c = 0; c <= a; ++c)
                    if (a * (a + 1) / 2 + c == qc) {
                        Pc = a;
                        Qc = c;
                    }
            cl.P = Pc;
            cl.Q = Qc;
            cl.ntiles = nt;
            cl.tiles = d_tiles + ex.off[k] + first;
            cl.stride = stride;
            cl.nsplit = cl.nchunk = 1;
            cl.kind = kinds ? kinds[k] : kind_all;
            cl.split_req = splits ? splits[k] : 0;
            OutArgs o = out;
            o.counters = dcnt + NCNT * qc;
            if (dump) o.dump = dump + (size_t)ex.off[k] * TILE * 12;
            const int grid = std::min(G, (grids && grids[k] > 0) ? grids[k] : G);  // cap; the launcher sizes it
            if (timing) cudaEventRecord(e0, st);
            cudaError_t e = kClassLaunchers[qc](r, grid, smem, st, d_mols, cl, o, boys);
            if (e != cudaSuccess) {
                cudaGetLastError();
                rc = TG_ECUDA;
                break;
            }
            ++launches;
            if (timing) {
                cudaEventRecord(e1, st);
                cudaEventSynchronize(e1);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (stats) (r ? stats->class_ms_fp32 : stats->class_ms)[qc] += ms;
            }
        }
    }
    return rc;
}

// fp64 / fp32 FMA peaks of the current device (FLOP/s): SMs x (2 | 128) FMA
// per clock per SM x 2 x the SM clock
void alu_peaks(double &p64, double &p32)
{
    int dev = 0, nsm = 0, khz = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev) != cudaSuccess) {
        cudaGetLastError();
        p64 = p32 = 0.0;
        return;
    }
    p64 = (double)nsm * 2.0 * 2.0 * khz * 1e3;
    p32 = (double)nsm * 128.0 * 2.0 * khz * 1e3;
}

// Autotuner of the class launches: for every (class, precision) list of ex
// with more than nsm tiles, time a sample of 2 to 4 x nsm tiles taken at a
// fixed stride over the whole list (whose tiles run from the costliest to
// the cheapest) and search the kernel form (thread, group,
// warp), the grid cap (1, 2 or 4 CTAs per SM) and the unit shape (bra
// primitive splits per tile: automatic, 1 or 4) one coordinate at a time
// from (form 1, 2 CTAs per SM, automatic splits): the
// fastest form, then the fastest grid cap for it, then the fastest split
// (7 timed launches per list).  Lists left untimed keep kinds[k] = 0 (the
// default form), grids[k] = 0 (the persistent grid) and splits[k] = 0.
// The sample launches write into d_part and d_cnt, which the caller clears
// afterwards.
int tune_lists(const Exec &ex, const MolDesc *d_mols, const uint4 *d_tiles, double *d_part,
               unsigned long long *d_cnt, const double *boys, int G, int nsm, cudaStream_t st, int *kinds,
               int *grids, int *splits)
{
    for (int k = 0; k < 2 * NQC; ++k) kinds[k] = grids[k] = splits[k] = 0;
    EventPair ev;
    TG_CUDA(ev.create());
    cudaEvent_t e0 = ev.a, e1 = ev.b;
    for (int k = 0; k < 2 * NQC; ++k) {
        const long long nt = ex.off[k + 1] - ex.off[k];
        if (nt <= nsm) continue;
        Exec sub;
        sub.natom_total = ex.natom_total;
        sub.natom_max = ex.natom_max;
        // the sample: every step-th tile of the list (2 to 4 x nsm tiles spread
        // over its whole cost range, through the tile-shard stride)
        const int step = (int)std::max<long long>(1, nt / (2LL * nsm));
        for (int j = 0; j < 2 * NQC + 1; ++j) sub.off[j] = j <= k ? 0 : nt;
        auto time_cfg = [&](int kind, int mult, int split, float &ms) -> int {
            std::vector<int> gr(2 * NQC, std::min(G, mult * nsm)), kd(2 * NQC, kind), sp(2 * NQC, split);
            int dummy = 0;
            cudaEventRecord(e0, st);
            int rc = launch_exec(sub, d_mols, d_tiles + ex.off[k], d_part, d_cnt, nullptr, boys, G, gr.data(),
                                 false, st, nullptr, dummy, kd.data(), 0, 0, step, sp.data());
            cudaEventRecord(e1, st);
            if (rc != TG_OK) return rc;
            TG_CUDA(cudaEventSynchronize(e1));
            ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            return TG_OK;
        };
        int bk = 1, bm = 2, bs = 0;
        float best = -1.f;
        for (int kind = 1; kind <= 3; ++kind) {
            float ms;
            const int rc = time_cfg(kind, bm, bs, ms);
            if (rc != TG_OK) return rc;
            if (best < 0.f || ms < best) best = ms, bk = kind;
        }
        for (int mult : {1, 4}) {
            float ms;
            const int rc = time_cfg(bk, mult, bs, ms);
            if (rc != TG_OK) return rc;
            if (ms < best) best = ms, bm = mult;
        }
        for (int split : {1, 4}) {
            float ms;
            const int rc = time_cfg(bk, bm, split, ms);
            if (rc != TG_OK) return rc;
            if (ms < best) best = ms, bs = split;
        }
        kinds[k] = bk;
        grids[k] = std::min(G, bm * nsm);
        splits[k] = bs;
    }
    return TG_OK;
}

void fill_stats(tg_stats *stats, const unsigned long long *hc, long long pairs, long long tiles, int launches, int G,
                int nops = 2)
{
    if (!stats) return;
    double f64 = 0.0, f32 = 0.0, ms64 = 0.0, ms32 = 0.0;
    for (int qc = 0; qc < NQC; ++qc) {
        double fpq, fp;
        class_flops(qc, nops, &fpq, &fp);
        f64 += fpq * (double)hc[NCNT * qc + 1] + fp * (double)hc[NCNT * qc + 4];
        f32 += fpq * (double)hc[NCNT * qc + 3] + fp * (double)hc[NCNT * qc + 5];
        ms64 += stats->class_ms[qc];
        ms32 += stats->class_ms_fp32[qc];
    }
    stats->fp64_flop = f64;
    stats->fp32_flop = f32;
    double p64 = 0.0, p32 = 0.0;
    if (ms64 > 0.0 || ms32 > 0.0) alu_peaks(p64, p32);
    stats->fp64_frac_peak = (ms64 > 0.0 && p64 > 0.0) ? f64 / (ms64 * 1e-3) / p64 : 0.0;
    stats->fp32_frac_peak = (ms32 > 0.0 && p32 > 0.0) ? f32 / (ms32 * 1e-3) / p32 : 0.0;
    long long q = 0, pq = 0, q32 = 0;
    for (int qc = 0; qc < NQC; ++qc) {
        stats->class_quartets[qc] = (long long)hc[NCNT * qc];
        stats->class_prim_quartets[qc] = (long long)hc[NCNT * qc + 1];
        stats->class_prim_quartets_fp32[qc] = (long long)hc[NCNT * qc + 3];
        stats->class_bra_prims[qc] = (long long)hc[NCNT * qc + 4];
        stats->class_bra_prims_fp32[qc] = (long long)hc[NCNT * qc + 5];
        q += (long long)hc[NCNT * qc];
        pq += (long long)hc[NCNT * qc + 1] + (long long)hc[NCNT * qc + 3];
        q32 += (long long)hc[NCNT * qc + 2];
    }
    stats->quartets = q;
    stats->prim_quartets = pq;
    stats->fp32_quartets = q32;
    stats->pairs = pairs;
    stats->tiles = tiles;
    stats->launches = launches;
    stats->grid = G;
}

}  // namespace

struct tg_batch;
extern "C" void tg_batch_destroy(tg_batch *bt);

struct tg_batch {
    int nmol = 0;
    std::vector<tg_basis *> bases;
    std::vector<Plan> plans;
    Exec ex;
    DevArena arena;
    MolDesc *d_mols = nullptr;
    uint4 *d_tiles = nullptr;
    double *d_part = nullptr, *d_grad = nullptr;
    unsigned long long *d_cnt = nullptr;
    std::vector<int> grids, kinds, splits;
    int G = 1;
    int device_ptrs = 0;
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    long long pairs = 0;
    int launches = 0;
    std::vector<int> atom_off;
};

extern "C" {

int tg_grad2e(const tg_basis *cb, int npair, const tg_pair *pairs, const tg_options *opt_in, double *grad,
              tg_stats *stats)
{
    auto t0 = std::chrono::steady_clock::now();
    tg_basis *b = const_cast<tg_basis *>(cb);
    if (!b || !pairs || !grad) return TG_EINVAL;
    tg_options opt;
    if (opt_in) opt = *opt_in;
    else tg_options_default(&opt);
    if (opt.precision == TG_MIXED_LEARNED && (!opt.router || !opt.router->trained)) return TG_EROUTER;
    cudaStream_t st = (cudaStream_t)opt.stream;
    Plan pl;
    int rc = make_plan(b, npair, pairs, opt, st, pl, false);
    if (rc != TG_OK) return rc;
    const int natom = b->natom;
    int launches = pl.launches;
    DevArena &V = b->ws2;
    double *d_part = V.take<double>((size_t)pl.G * 3 * natom);
    MolDesc *d_mol = V.take<MolDesc>(1);
    // the screened tile lists, routed and split per (class, precision), built on the device
    DevTiles dt;
    rc = device_tiles(b, pl, opt, st, dt, launches);
    if (rc != TG_OK) return rc;
    const size_t ntl = (size_t)dt.ntiles;
    Exec ex;
    for (int k = 0; k <= 2 * NQC; ++k) ex.off[k] = dt.off[k];
    ex.natom_total = ex.natom_max = natom;
    const uint4 *d_tiles = dt.tiles;
    const MolDesc md = make_desc(pl, 0);
    TG_CUDA(cudaMemcpyAsync(d_mol, &md, sizeof(MolDesc), cudaMemcpyHostToDevice, st));
    // autotune = 1: the per-list launch choices of the basis's first tuned
    // call; autotune = 2: tune again on this call and keep the new choices
    int kd[2 * NQC], gr[2 * NQC], sp[2 * NQC];
    const bool tune = opt.autotune == 1 || opt.autotune == 2;
    if (tune) {
        if (!b->tuned || opt.autotune == 2) {
            rc = tune_lists(ex, d_mol, d_tiles, d_part, pl.dcnt, b->d_boys, pl.G, b->nsm, st, b->tune_kind,
                            b->tune_grid, b->tune_split);
            if (rc != TG_OK) return rc;
            b->tuned = true;
        }
        for (int k = 0; k < 2 * NQC; ++k) {
            kd[k] = b->tune_kind[k] ? b->tune_kind[k] : opt.kernel_kind;
            gr[k] = b->tune_grid[k];
            sp[k] = b->tune_split[k];
        }
    }
    TG_CUDA(cudaMemsetAsync(d_part, 0, sizeof(double) * (size_t)pl.G * 3 * natom, st));
    TG_CUDA(cudaMemsetAsync(pl.dcnt, 0, sizeof(unsigned long long) * NCNT * NQC, st));
    if (stats)
        for (int qc = 0; qc < NQC; ++qc) stats->class_ms[qc] = stats->class_ms_fp32[qc] = 0.0;
    const double plan_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    // (a tile shard is already in the lists)
    rc = launch_exec(ex, d_mol, d_tiles, d_part, pl.dcnt, nullptr, b->d_boys, pl.G, tune ? gr : nullptr,
                     opt.timing != 0, st, stats, launches, tune ? kd : nullptr, opt.kernel_kind, 0, 1,
                     tune ? sp : nullptr);
    if (rc != TG_OK) return rc;
    k_reduce<<<(3 * natom + 127) / 128, 128, 0, st>>>(3 * natom, pl.G, d_part, pl.dgrad);
    ++launches;
    TG_CUDA(cudaGetLastError());
    unsigned long long hc[NCNT * NQC];
    TG_CUDA(cudaMemcpyAsync(hc, pl.dcnt, sizeof(hc), cudaMemcpyDeviceToHost, st));
    TG_CUDA(cudaMemcpyAsync(grad, pl.dgrad, sizeof(double) * 3 * natom,
                            opt.device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
    TG_CUDA(cudaStreamSynchronize(st));
    if (stats) {
        fill_stats(stats, hc, pl.npairs_kept, (long long)ntl, launches, pl.G, pl.den.use_lr ? 2 : 1);
        stats->plan_ms = plan_ms;
        stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    return TG_OK;
}

int tg_grad2e_sph(const tg_basis *cb, int npair, const tg_pair *pairs, const tg_options *opt_in, double *grad,
                  tg_stats *stats)
{
    tg_basis *b = const_cast<tg_basis *>(cb);
    if (!b || !pairs || !grad) return TG_EINVAL;
    tg_options opt;
    if (opt_in) opt = *opt_in;
    else tg_options_default(&opt);
    // every argument is checked before the first CUDA call
    double om = 0.0;
    int lr = 0;
    const int rc0 = check_pairs(npair, pairs, opt, om, lr);
    if (rc0 != TG_OK) return rc0;
    if (opt.precision == TG_MIXED_LEARNED && (!opt.router || !opt.router->trained)) return TG_EROUTER;
    cudaStream_t st = (cudaStream_t)opt.stream;
    const size_t nbf = (size_t)b->nbf, nsph = (size_t)b->nsph, natom = (size_t)b->natom;
    const int nup = opt.device_ptrs ? 0 : 2 * npair;
    const size_t need = al(sizeof(double) * nsph * nsph) * nup + al(sizeof(double) * nbf * nbf) * 2 * npair +
                        al(sizeof(int) * nbf) + al(sizeof(double) * 3 * natom) + 4096;
    DevArena &W = b->ws6;
    TG_CUDA(W.reserve(need));
    W.used = 0;
    int *d_cmap = W.take<int>(nbf);
    double *d_grad = W.take<double>(3 * natom);
    TG_CUDA(cudaMemcpyAsync(d_cmap, b->cmap.data(), sizeof(int) * nbf, cudaMemcpyHostToDevice, st));
    tg_pair cp[TG_MAX_PAIRS];
    const unsigned gs = (unsigned)((nbf * nbf + 255) / 256);
    for (int p = 0; p < npair; ++p) {
        const double *src[2] = {pairs[p].A, pairs[p].B};
        double *dst[2];
        for (int k = 0; k < 2; ++k) {
            const double *a = src[k];
            if (!opt.device_ptrs) {
                double *up = W.take<double>(nsph * nsph);
                TG_CUDA(cudaMemcpyAsync(up, a, sizeof(double) * nsph * nsph, cudaMemcpyHostToDevice, st));
                a = up;
            }
            dst[k] = W.take<double>(nbf * nbf);
            k_sph_to_cart<<<gs, 256, 0, st>>>((int)nbf, (int)nsph, d_cmap, a, dst[k]);
            TG_CUDA(cudaGetLastError());
        }
        cp[p] = pairs[p];
        cp[p].A = dst[0];
        cp[p].B = dst[1];
    }
    tg_options o2 = opt;
    o2.device_ptrs = 1;
    int rc = tg_grad2e(cb, npair, cp, &o2, d_grad, stats);
    if (rc != TG_OK) return rc;
    TG_CUDA(cudaMemcpyAsync(grad, d_grad, sizeof(double) * 3 * natom,
                            opt.device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
    TG_CUDA(cudaStreamSynchronize(st));
    if (stats) stats->launches += 2 * npair;
    return TG_OK;
}

int tg_fock2e(const tg_basis *cb, int npair, const tg_fpair *fpairs, const tg_options *opt_in, double *F,
              tg_stats *stats)
{
    auto t0 = std::chrono::steady_clock::now();
    tg_basis *b = const_cast<tg_basis *>(cb);
    if (!b || !fpairs || !F) return TG_EINVAL;
    tg_options opt;
    if (opt_in) opt = *opt_in;
    else tg_options_default(&opt);
    if (npair < 1) return TG_EINVAL;
    if (npair > TG_MAX_PAIRS) return TG_EUNSUPPORTED;
    if (!(opt.screen_tol >= 0.0) || !std::isfinite(opt.screen_tol)) return TG_EINVAL;
    if (opt.precision != TG_FP64 || opt.nranks != 1 || opt.rank != 0) return TG_EUNSUPPORTED;
    if (opt.class_mask >> NQC) return TG_EINVAL;
    for (int r : opt.reserved)
        if (r != 0) return TG_EINVAL;
    double omega = 0.0;
    int use_lr = 0;
    for (int p = 0; p < npair; ++p) {
        const tg_fpair &q = fpairs[p];
        if (!q.B) return TG_EINVAL;
        if (!std::isfinite(q.c_J) || !std::isfinite(q.c_K) || !std::isfinite(q.c_K_lr) || std::isnan(q.omega))
            return TG_EINVAL;
        if (q.c_K_lr != 0.0 && q.omega > 0.0) {
            if (use_lr && q.omega != omega) return TG_EUNSUPPORTED;
            use_lr = 1;
            omega = q.omega;
        }
    }
    cudaStream_t st = (cudaStream_t)opt.stream;
    TG_CUDA(cudaSetDevice(b->device));
    const int nbf = b->nbf, natom = b->natom;
    const size_t nbf2 = (size_t)nbf * nbf;
    // densities (device copies of host matrices), the combined matrices and F
    DevArena &Z = b->ws5;
    const int nup = opt.device_ptrs ? 0 : npair;
    TG_CUDA(Z.reserve(al(sizeof(double) * nbf2) * (nup + 4) + 4096));
    Z.used = 0;
    DensArgs dn;
    std::memset(&dn, 0, sizeof(dn));
    dn.npair = npair;
    dn.nbf = nbf;
    for (int p = 0; p < npair; ++p) {
        if (opt.device_ptrs) {
            dn.A[p] = fpairs[p].B;
        } else {
            double *d = Z.take<double>(nbf2);
            TG_CUDA(cudaMemcpyAsync(d, fpairs[p].B, sizeof(double) * nbf2, cudaMemcpyHostToDevice, st));
            dn.A[p] = d;
        }
        dn.cJ[p] = fpairs[p].c_J;
        dn.cK[p] = fpairs[p].c_K;
        dn.cKlr[p] = fpairs[p].omega > 0.0 ? fpairs[p].c_K_lr : 0.0;
    }
    double *SJ = Z.take<double>(nbf2), *BK = Z.take<double>(nbf2), *BL = Z.take<double>(nbf2);
    double *dF = Z.take<double>(nbf2);
    const unsigned gs = (unsigned)((nbf2 + 255) / 256);
    k_fock_combine<<<gs, 256, 0, st>>>(nbf, dn, SJ, BK, BL);
    TG_CUDA(cudaMemsetAsync(dF, 0, sizeof(double) * nbf2, st));
    TG_CUDA(cudaGetLastError());
    // plan over the combined matrices: M = max(|S_J|, |B_K|, |B_lr|) per shell block
    tg_pair pseudo[2];
    pseudo[0] = {SJ, BK, 1.0, 0.0, 0.0, 0.0};
    pseudo[1] = {BL, BL, 1.0, 0.0, 0.0, 0.0};
    tg_options po = opt;
    po.device_ptrs = 1;
    po.precision = TG_FP64;
    po.nranks = 1;
    po.rank = 0;
    Plan pl;
    int rc = make_plan(b, 2, pseudo, po, st, pl, false, true);
    if (rc != TG_OK) return rc;
    pl.den.use_lr = use_lr;
    pl.den.omega = omega;
    pl.scr.scale = pl.scale;
    int launches = pl.launches + 1;
    DevArena &V = b->ws2;
    MolDesc *d_mol = V.take<MolDesc>(1);
    DevTiles dt;
    rc = device_tiles(b, pl, po, st, dt, launches);
    if (rc != TG_OK) return rc;
    const MolDesc md = make_desc(pl, 0);
    TG_CUDA(cudaMemcpyAsync(d_mol, &md, sizeof(MolDesc), cudaMemcpyHostToDevice, st));
    TG_CUDA(cudaMemsetAsync(pl.dcnt, 0, sizeof(unsigned long long) * NCNT * NQC, st));
    if (stats)
        for (int qc = 0; qc < NQC; ++qc) stats->class_ms[qc] = stats->class_ms_fp32[qc] = 0.0;
    const double plan_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    EventPair ev;
    if (opt.timing) TG_CUDA(ev.create());
    for (int qc = 0; qc < NQC; ++qc) {
        const long long nt = dt.off[2 * qc + 1] - dt.off[2 * qc];
        if (nt <= 0) continue;
        ClassLaunch cl;
        std::memset(&cl, 0, sizeof(cl));
        cl.P = pl.qc_P[qc];
        cl.Q = pl.qc_Q[qc];
        cl.ntiles = nt;
        cl.tiles = dt.tiles + dt.off[2 * qc];
        cl.stride = 1;
        cl.nsplit = cl.nchunk = 1;
        OutArgs o;
        std::memset(&o, 0, sizeof(o));
        o.counters = pl.dcnt + NCNT * qc;
        o.natom_total = o.natom_max = natom;
        o.fock = dF;
        if (opt.timing) cudaEventRecord(ev.a, st);
        cudaError_t e = kFockLaunchers[qc](pl.G, st, d_mol, cl, o, b->d_boys);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return TG_ECUDA;
        }
        ++launches;
        if (opt.timing) {
            cudaEventRecord(ev.b, st);
            cudaEventSynchronize(ev.b);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, ev.a, ev.b);
            if (stats) stats->class_ms[qc] += ms;
        }
    }
    unsigned long long hc[NCNT * NQC];
    TG_CUDA(cudaMemcpyAsync(hc, pl.dcnt, sizeof(hc), cudaMemcpyDeviceToHost, st));
    TG_CUDA(cudaMemcpyAsync(F, dF, sizeof(double) * nbf2,
                            opt.device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
    TG_CUDA(cudaStreamSynchronize(st));
    if (stats) {
        fill_stats(stats, hc, pl.npairs_kept, dt.ntiles, launches, pl.G, use_lr ? 2 : 1);
        stats->fp64_flop = 0.0;  // the gradient's FLOP count does not apply
        stats->fp64_frac_peak = 0.0;
        stats->plan_ms = plan_ms;
        stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    return TG_OK;
}

int tg_tile_samples(const tg_basis *cb, int npair, const tg_pair *pairs, const tg_options *opt_in, int stride,
                    int cap, float *features, float *target, float *err32, int *n_out)
{
    tg_basis *b = const_cast<tg_basis *>(cb);
    if (!b || !pairs || !features || !target || !err32 || !n_out || stride < 1 || cap < 0) return TG_EINVAL;
    tg_options opt;
    if (opt_in) opt = *opt_in;
    else tg_options_default(&opt);
    cudaStream_t st = (cudaStream_t)opt.stream;
    Plan pl;
    int rc = make_plan(b, npair, pairs, opt, st, pl);
    if (rc != TG_OK) return rc;
    std::vector<size_t> pick;
    for (size_t i = 0; i < pl.tiles.size() && (int)pick.size() < cap; i += stride) pick.push_back(i);
    const size_t n = pick.size();
    *n_out = (int)n;
    if (!n) return TG_OK;
    DevArena &V = b->ws2;
    const size_t need = V.used + al(sizeof(uint4) * n) + al(sizeof(TileRef) * n) + al(sizeof(float) * n * (NFEAT + 1)) +
                        2 * al(sizeof(double) * n * TILE * 12) + al(sizeof(double) * (size_t)pl.G * 3 * b->natom) +
                        al(sizeof(MolDesc)) + 8192;
    if (need > V.cap) {
        // grow the plan arena, then rebuild the plan inside it
        TG_CUDA(cudaStreamSynchronize(st));
        V.release();
        TG_CUDA(V.reserve(need + need / 4));
        return tg_tile_samples(cb, npair, pairs, opt_in, stride, cap, features, target, err32, n_out);
    }
    uint4 *d_tiles = V.take<uint4>(n);
    TileRef *d_ref = V.take<TileRef>(n);
    float *d_feat = V.take<float>(n * NFEAT);
    float *d_pred = V.take<float>(n);
    double *d64 = V.take<double>(n * TILE * 12);
    double *d32 = V.take<double>(n * TILE * 12);
    double *d_part = V.take<double>((size_t)pl.G * 3 * b->natom);
    MolDesc *d_mol = V.take<MolDesc>(1);
    int launches = 0;
    std::vector<float> feat;
    rc = predict_tiles(b, pl, nullptr, pick, st, d_ref, d_feat, d_pred, nullptr, &feat, launches);
    if (rc != TG_OK) return rc;
    const MolDesc md = make_desc(pl, 0);
    TG_CUDA(cudaMemcpyAsync(d_mol, &md, sizeof(MolDesc), cudaMemcpyHostToDevice, st));
    // samples in class order so every launch covers a contiguous dump range
    std::vector<std::vector<size_t>> subset(1, pick);
    for (int r = 0; r < 2; ++r) {
        std::vector<std::vector<uint8_t>> routes(1, std::vector<uint8_t>(pl.tiles.size(), (uint8_t)r));
        Exec ex;
        build_exec({&pl}, routes, &subset, ex);
        ex.natom_total = ex.natom_max = b->natom;
        TG_CUDA(cudaMemcpyAsync(d_tiles, ex.tiles.data(), sizeof(uint4) * ex.tiles.size(), cudaMemcpyHostToDevice, st));
        TG_CUDA(cudaMemsetAsync(pl.dcnt, 0, sizeof(unsigned long long) * NCNT * NQC, st));
        // the dump is written at list positions; lists are class-major with r fixed,
        // so positions run over the samples in class order
        rc = launch_exec(ex, d_mol, d_tiles, d_part, pl.dcnt, r ? d32 : d64, b->d_boys, pl.G, nullptr, false, st,
                         nullptr, launches);
        if (rc != TG_OK) return rc;
        TG_CUDA(cudaStreamSynchronize(st));
    }
    std::vector<size_t> pos(pl.tiles.size(), 0);
    {
        size_t p = 0;
        for (int qc = 0; qc < NQC; ++qc)
            for (size_t i : pick)
                if (pl.tiles[i].qc == qc) pos[i] = p++;
    }
    std::vector<double> h64(n * TILE * 12), h32(n * TILE * 12);
    TG_CUDA(cudaMemcpy(h64.data(), d64, sizeof(double) * h64.size(), cudaMemcpyDeviceToHost));
    TG_CUDA(cudaMemcpy(h32.data(), d32, sizeof(double) * h32.size(), cudaMemcpyDeviceToHost));
    // a tile's contribution to the gradient: per atom and component, the sum
    // over its quartets; target = the largest |sum| (fp64), err32 = the
    // largest |sum(fp32) - sum(fp64)|
    std::vector<double> s64(3 * (size_t)b->natom), s32(3 * (size_t)b->natom);
    for (size_t k = 0; k < n; ++k) {
        const HostTile &t = pl.tiles[pick[k]];
        const int P = pl.qc_P[t.qc], Qc = pl.qc_Q[t.qc];
        std::fill(s64.begin(), s64.end(), 0.0);
        std::fill(s32.begin(), s32.end(), 0.0);
        const size_t p = pos[pick[k]];
        for (int q = 0; q < TILE; ++q) {
            const int bi = t.bt * TB + q / TK, ki = t.kt * TK + q % TK;
            if (bi >= (int)pl.cls[P].size() || ki >= (int)pl.cls[Qc].size()) continue;
            const HostPair &u = pl.cls[P][bi], &v = pl.cls[Qc][ki];
            const int at[4] = {b->sh_atom[u.sa], b->sh_atom[u.sb], b->sh_atom[v.sa], b->sh_atom[v.sb]};
            const double *g64 = &h64[(p * TILE + q) * 12], *g32 = &h32[(p * TILE + q) * 12];
            for (int X = 0; X < 4; ++X)
                for (int i = 0; i < 3; ++i) {
                    s64[at[X] * 3 + i] += g64[X * 3 + i];
                    s32[at[X] * 3 + i] += g32[X * 3 + i];
                }
        }
        double mx = 0.0, me = 0.0;
        for (size_t j = 0; j < s64.size(); ++j) {
            mx = std::max(mx, std::fabs(s64[j]));
            me = std::max(me, std::fabs(s32[j] - s64[j]));
        }
        target[k] = (float)std::log10(mx + 1e-30);
        err32[k] = (float)std::log10(me + 1e-30);
        for (int f = 0; f < NFEAT; ++f) features[k * NFEAT + f] = feat[k * NFEAT + f];
    }
    return TG_OK;
}

// ------------------------------------------------------------------ batch
// Plan once, replay many: every molecule of the batch is planned (screening,
// class sort, routing) at creation; one persistent launch per (class,
// precision) then covers the tiles of all molecules, and the whole launch
// sequence is captured in a CUDA graph that tg_batch_run replays.
int tg_batch_create(int nmol, const tg_basis *const *bases, const int *npair, const tg_pair *const *pairs,
                    const tg_options *opt_in, tg_batch **out)
{
    if (!out || nmol < 1 || !bases || !npair || !pairs) return TG_EINVAL;
    *out = nullptr;
    tg_options opt;
    if (opt_in) opt = *opt_in;
    else tg_options_default(&opt);
    if (opt.precision == TG_MIXED_LEARNED && (!opt.router || !opt.router->trained)) return TG_EROUTER;
    for (int m = 0; m < nmol; ++m) {
        if (!bases[m]) return TG_EINVAL;
        for (int k = 0; k < m; ++k)
            if (bases[k] == bases[m]) return TG_EINVAL;  // a basis holds one plan at a time
    }
    tg_batch *bt = new (std::nothrow) tg_batch();
    if (!bt) return TG_ENOMEM;
    std::unique_ptr<tg_batch, void (*)(tg_batch *)> guard(bt, [](tg_batch *x) { tg_batch_destroy(x); });
    bt->nmol = nmol;
    bt->plans.resize(nmol);
    bt->device_ptrs = opt.device_ptrs;
    cudaStream_t st = (cudaStream_t)opt.stream;
    std::vector<std::vector<uint8_t>> routes(nmol);
    std::vector<const Plan *> pp(nmol);
    int natom_total = 0, natom_max = 0, G = 1;
    for (int m = 0; m < nmol; ++m) {
        tg_basis *b = const_cast<tg_basis *>(bases[m]);
        bt->bases.push_back(b);
        Plan &pl = bt->plans[m];
        int rc = make_plan(b, npair[m], pairs[m], opt, st, pl);
        if (rc != TG_OK) return rc;
        bt->launches += pl.launches;
        const size_t ntl = std::max<size_t>(pl.tiles.size(), 1);
        DevArena &V = b->ws2;
        TileRef *d_ref = V.take<TileRef>(ntl);
        float *d_feat = V.take<float>(ntl * NFEAT);
        float *d_pred = V.take<float>(ntl);
        rc = compute_route(b, pl, opt, st, d_ref, d_feat, d_pred, routes[m], bt->launches);
        if (rc != TG_OK) return rc;
        bt->atom_off.push_back(natom_total);
        natom_total += b->natom;
        natom_max = std::max(natom_max, b->natom);
        G = std::max(G, pl.G);
        bt->pairs += pl.npairs_kept;
        pp[m] = &pl;
    }
    build_exec(pp, routes, nullptr, bt->ex);
    bt->ex.natom_total = natom_total;
    bt->ex.natom_max = natom_max;
    bt->G = G;
    const size_t ntl = std::max<size_t>(bt->ex.tiles.size(), 1);
    const size_t need = al(sizeof(MolDesc) * nmol) + al(sizeof(uint4) * ntl) +
                        al(sizeof(double) * (size_t)G * 3 * natom_total) + al(sizeof(double) * 3 * natom_total) +
                        al(sizeof(unsigned long long) * NCNT * NQC) + 4096;
    TG_CUDA(bt->arena.reserve(need));
    bt->arena.used = 0;
    bt->d_mols = bt->arena.take<MolDesc>(nmol);
    bt->d_tiles = bt->arena.take<uint4>(ntl);
    bt->d_part = bt->arena.take<double>((size_t)G * 3 * natom_total);
    bt->d_grad = bt->arena.take<double>(3 * natom_total);
    bt->d_cnt = bt->arena.take<unsigned long long>(NCNT * NQC);
    std::vector<MolDesc> mds(nmol);
    for (int m = 0; m < nmol; ++m) mds[m] = make_desc(bt->plans[m], bt->atom_off[m]);
    TG_CUDA(cudaMemcpy(bt->d_mols, mds.data(), sizeof(MolDesc) * nmol, cudaMemcpyHostToDevice));
    if (!bt->ex.tiles.empty())
        TG_CUDA(cudaMemcpy(bt->d_tiles, bt->ex.tiles.data(), sizeof(uint4) * bt->ex.tiles.size(),
                           cudaMemcpyHostToDevice));
    const double *boys = bt->bases[0]->d_boys;

    // ---- autotune every (class, precision) list (tune_lists)
    bt->grids.assign(2 * NQC, G);
    bt->kinds.assign(2 * NQC, opt.kernel_kind);
    bt->splits.assign(2 * NQC, 0);
    const int nsm = std::max(1, bt->bases[0]->nsm);
    if (opt.autotune == 1 || opt.autotune == 2) {
        int kd[2 * NQC], gr[2 * NQC], sp[2 * NQC];
        const int rc = tune_lists(bt->ex, bt->d_mols, bt->d_tiles, bt->d_part, bt->d_cnt, boys, G, nsm, st, kd, gr,
                                  sp);
        if (rc != TG_OK) return rc;
        for (int k = 0; k < 2 * NQC; ++k) {
            if (kd[k]) bt->kinds[k] = kd[k];
            if (gr[k]) bt->grids[k] = gr[k];
            bt->splits[k] = sp[k];
        }
    }
    // the partial slabs must cover the largest tuned grid
    if ((size_t)G * 3 * natom_total > (size_t)bt->plans[0].G * 3 * natom_total) {
        // re-carve with the larger slab count
        bt->arena.release();
        const size_t need2 = al(sizeof(MolDesc) * nmol) + al(sizeof(uint4) * ntl) +
                             al(sizeof(double) * (size_t)G * 3 * natom_total) + al(sizeof(double) * 3 * natom_total) +
                             al(sizeof(unsigned long long) * NCNT * NQC) + 4096;
        TG_CUDA(bt->arena.reserve(need2));
        bt->arena.used = 0;
        bt->d_mols = bt->arena.take<MolDesc>(nmol);
        bt->d_tiles = bt->arena.take<uint4>(ntl);
        bt->d_part = bt->arena.take<double>((size_t)G * 3 * natom_total);
        bt->d_grad = bt->arena.take<double>(3 * natom_total);
        bt->d_cnt = bt->arena.take<unsigned long long>(NCNT * NQC);
        TG_CUDA(cudaMemcpy(bt->d_mols, mds.data(), sizeof(MolDesc) * nmol, cudaMemcpyHostToDevice));
        if (!bt->ex.tiles.empty())
            TG_CUDA(cudaMemcpy(bt->d_tiles, bt->ex.tiles.data(), sizeof(uint4) * bt->ex.tiles.size(),
                               cudaMemcpyHostToDevice));
    }

    // ---- capture the launch sequence once (a run first sets kernel attributes)
    TG_CUDA(cudaStreamCreateWithFlags(&bt->cap, cudaStreamNonBlocking));
    for (int pass = 0; pass < 2; ++pass) {
        if (pass == 1) TG_CUDA(cudaStreamBeginCapture(bt->cap, cudaStreamCaptureModeThreadLocal));
        int n = 0;
        cudaMemsetAsync(bt->d_part, 0, sizeof(double) * (size_t)G * 3 * natom_total, bt->cap);
        cudaMemsetAsync(bt->d_cnt, 0, sizeof(unsigned long long) * NCNT * NQC, bt->cap);
        int rc = launch_exec(bt->ex, bt->d_mols, bt->d_tiles, bt->d_part, bt->d_cnt, nullptr, boys, G,
                             bt->grids.data(), false, bt->cap, nullptr, n, bt->kinds.data(), 0, 0, 1,
                             bt->splits.data());
        k_reduce<<<(3 * natom_total + 127) / 128, 128, 0, bt->cap>>>(3 * natom_total, G, bt->d_part, bt->d_grad);
        ++n;
        if (pass == 1) {
            cudaError_t e = cudaStreamEndCapture(bt->cap, &bt->graph);
            if (rc != TG_OK) return rc;
            TG_CUDA(e);
            TG_CUDA(cudaGraphInstantiate(&bt->gexec, bt->graph, 0));
            bt->launches = n;
        } else {
            if (rc != TG_OK) return rc;
            TG_CUDA(cudaStreamSynchronize(bt->cap));
        }
    }
    *out = guard.release();
    return TG_OK;
}

int tg_batch_run(tg_batch *bt, double *const *grads, const tg_options *opt_in, tg_stats *stats)
{
    if (!bt || !grads) return TG_EINVAL;
    auto t0 = std::chrono::steady_clock::now();
    tg_options opt;
    if (opt_in) opt = *opt_in;
    else tg_options_default(&opt);
    cudaStream_t st = (cudaStream_t)opt.stream;
    // every argument is checked before the first CUDA call
    for (int m = 0; m < bt->nmol; ++m)
        if (!grads[m]) return TG_EINVAL;
    TG_CUDA(cudaGraphLaunch(bt->gexec, st));
    unsigned long long hc[NCNT * NQC];
    TG_CUDA(cudaMemcpyAsync(hc, bt->d_cnt, sizeof(hc), cudaMemcpyDeviceToHost, st));
    for (int m = 0; m < bt->nmol; ++m) {
        TG_CUDA(cudaMemcpyAsync(grads[m], bt->d_grad + 3 * (size_t)bt->atom_off[m],
                                sizeof(double) * 3 * bt->bases[m]->natom,
                                opt.device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
    }
    TG_CUDA(cudaStreamSynchronize(st));
    if (stats) {
        for (int qc = 0; qc < NQC; ++qc) stats->class_ms[qc] = stats->class_ms_fp32[qc] = 0.0;
        int nops = 1;
        for (const Plan &pl : bt->plans)
            if (pl.den.use_lr) nops = 2;
        fill_stats(stats, hc, bt->pairs, (long long)bt->ex.tiles.size(), bt->launches, bt->G, nops);
        stats->plan_ms = 0.0;  // planned at tg_batch_create
        stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    return TG_OK;
}

void tg_batch_destroy(tg_batch *bt)
{
    if (!bt) return;
    if (bt->gexec) cudaGraphExecDestroy(bt->gexec);
    if (bt->graph) cudaGraphDestroy(bt->graph);
    if (bt->cap) cudaStreamDestroy(bt->cap);
    bt->arena.release();
    delete bt;
}

}  // extern "C"


// ------------------------------------------------------------------ router
namespace {

uint64_t splitmix64(uint64_t &x)
{
    uint64_t z = (x += 0x9e3779b97f4a7c15ULL);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

struct DevBufs {
    std::vector<void *> ptrs;
    ~DevBufs()
    {
        for (void *p : ptrs) cudaFree(p);
    }
    template <typename T>
    cudaError_t alloc(T **p, size_t n)
    {
        cudaError_t e = cudaMalloc((void **)p, sizeof(T) * std::max<size_t>(n, 1));
        if (e == cudaSuccess) ptrs.push_back(*p);
        return e;
    }
};

}  // namespace

extern "C" {

int tg_router_nparam(void) { return NPARAM; }

int tg_router_create(unsigned long long seed, tg_router **out)
{
    if (!out) return TG_EINVAL;
    tg_router *r = new (std::nothrow) tg_router();
    if (!r) return TG_ENOMEM;
    uint64_t st = seed;
    auto uni = [&]() { return (double)(splitmix64(st) >> 11) * (1.0 / 9007199254740992.0); };
    // Xavier-uniform weights, zero biases
    int o = 0;
    const int fan[3][2] = {{NFEAT, NH}, {NH, NH}, {NH, 1}};
    for (int layer = 0; layer < 3; ++layer) {
        const int fin = fan[layer][0], fout = fan[layer][1];
        const double a = std::sqrt(6.0 / (fin + fout));
        for (int k = 0; k < fin * fout; ++k) r->params[o++] = (float)((2.0 * uni() - 1.0) * a);
        for (int k = 0; k < fout; ++k) r->params[o++] = 0.f;
    }
    for (int j = 0; j < NFEAT; ++j) {
        r->mu[j] = 0.f;
        r->sd[j] = 1.f;
    }
    *out = r;
    return TG_OK;
}

void tg_router_destroy(tg_router *r) { delete r; }

int tg_router_get(const tg_router *r, float *params, float *mu, float *sd, float *calib)
{
    if (!r) return TG_EINVAL;
    if (params) std::memcpy(params, r->params, sizeof(r->params));
    if (mu) std::memcpy(mu, r->mu, sizeof(r->mu));
    if (sd) std::memcpy(sd, r->sd, sizeof(r->sd));
    if (calib) {
        calib[0] = r->margin;
        calib[1] = r->eps_rel;
        calib[2] = (float)r->trained;
    }
    return TG_OK;
}

int tg_router_set(tg_router *r, const float *params, const float *mu, const float *sd, const float *calib)
{
    if (!r) return TG_EINVAL;
    // validate everything first: on error the router is left as it was
    if (params)
        for (int k = 0; k < NPARAM; ++k)
            if (!std::isfinite(params[k])) return TG_EINVAL;
    if (mu)
        for (int j = 0; j < NFEAT; ++j)
            if (!std::isfinite(mu[j])) return TG_EINVAL;
    if (sd)
        for (int j = 0; j < NFEAT; ++j)
            if (!(sd[j] > 0.f) || !std::isfinite(sd[j])) return TG_EINVAL;
    if (calib && (!std::isfinite(calib[0]) || !(calib[1] >= 0.f) || !std::isfinite(calib[1]))) return TG_EINVAL;
    if (params) std::memcpy(r->params, params, sizeof(r->params));
    if (mu) std::memcpy(r->mu, mu, sizeof(r->mu));
    if (sd) std::memcpy(r->sd, sd, sizeof(r->sd));
    if (calib) {
        r->margin = calib[0];
        r->eps_rel = calib[1];
        r->trained = calib[2] != 0.f;
    }
    return TG_OK;
}

static int router_loss_grad_dev(const tg_router *r, int n, const float *dX, const float *dy, const float *dmu,
                                const float *dsd, const float *dparams, float q, float *dgrad, float *dloss,
                                float *gpart, float *lpart)
{
    const int nblk = (n + TRB - 1) / TRB;
    // the dynamic shared-memory limit is a per-device attribute of the kernel
    constexpr int kMaxDev = 64;
    static bool attr[kMaxDev] = {false};
    int dev = 0;
    TG_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDev) return TG_ECUDA;
    if (!attr[dev]) {
        TG_CUDA(cudaFuncSetAttribute(k_mlp_fwd_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)fwd_bwd_smem()));
        attr[dev] = true;
    }
    k_mlp_fwd_bwd<<<nblk, TRB, fwd_bwd_smem()>>>(n, dX, dy, dmu, dsd, dparams, q, gpart, lpart);
    k_sum_partials<<<(NPARAM + 127) / 128, 128>>>(nblk, NPARAM, gpart, dgrad);
    k_sum_partials<<<1, 32>>>(nblk, 1, lpart, dloss);
    TG_CUDA(cudaGetLastError());
    (void)r;
    return TG_OK;
}

// Training on the GPU: feature standardisation, then `epochs` full-batch
// Adam steps on the expectile loss (quantile q) with a cosine learning-rate
// decay.  loss_hist (nullable, epochs floats) receives the loss before each step.
int tg_router_train(tg_router *r, int n, const float *X, const float *y, int epochs, float lr, float q,
                    float *loss_hist)
{
    if (!r || n < 1 || !X || !y || epochs < 1 || !(lr > 0.f) || !(q > 0.f && q < 1.f)) return TG_EINVAL;
    DevBufs B;
    float *dX, *dy, *dmu, *dsd, *dp, *dm, *dv, *dg, *dl, *gpart, *lpart;
    const int nblk = (n + TRB - 1) / TRB;
    TG_CUDA(B.alloc(&dX, (size_t)n * NFEAT));
    TG_CUDA(B.alloc(&dy, n));
    TG_CUDA(B.alloc(&dmu, NFEAT));
    TG_CUDA(B.alloc(&dsd, NFEAT));
    TG_CUDA(B.alloc(&dp, NPARAM));
    TG_CUDA(B.alloc(&dm, NPARAM));
    TG_CUDA(B.alloc(&dv, NPARAM));
    TG_CUDA(B.alloc(&dg, NPARAM));
    TG_CUDA(B.alloc(&dl, epochs));
    TG_CUDA(B.alloc(&gpart, (size_t)nblk * NPARAM));
    TG_CUDA(B.alloc(&lpart, nblk));
    TG_CUDA(cudaMemcpy(dX, X, sizeof(float) * n * NFEAT, cudaMemcpyHostToDevice));
    TG_CUDA(cudaMemcpy(dy, y, sizeof(float) * n, cudaMemcpyHostToDevice));
    TG_CUDA(cudaMemcpy(dp, r->params, sizeof(float) * NPARAM, cudaMemcpyHostToDevice));
    TG_CUDA(cudaMemset(dm, 0, sizeof(float) * NPARAM));
    TG_CUDA(cudaMemset(dv, 0, sizeof(float) * NPARAM));
    k_feature_stats<<<1, 32>>>(n, dX, dmu, dsd);
    TG_CUDA(cudaGetLastError());
    for (int ep = 0; ep < epochs; ++ep) {
        int rc = router_loss_grad_dev(r, n, dX, dy, dmu, dsd, dp, q, dg, dl + ep, gpart, lpart);
        if (rc != TG_OK) return rc;
        const float lr_t = lr * (0.05f + 0.95f * 0.5f * (1.f + std::cos(3.14159265f * ep / epochs)));
        k_adam<<<(NPARAM + 127) / 128, 128>>>(NPARAM, dp, dg, dm, dv, lr_t, 0.9f, 0.999f, 1e-8f, ep + 1);
    }
    TG_CUDA(cudaGetLastError());
    TG_CUDA(cudaMemcpy(r->params, dp, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost));
    TG_CUDA(cudaMemcpy(r->mu, dmu, sizeof(float) * NFEAT, cudaMemcpyDeviceToHost));
    TG_CUDA(cudaMemcpy(r->sd, dsd, sizeof(float) * NFEAT, cudaMemcpyDeviceToHost));
    if (loss_hist) TG_CUDA(cudaMemcpy(loss_hist, dl, sizeof(float) * epochs, cudaMemcpyDeviceToHost));
    return TG_OK;
}

// Loss and parameter gradient of the current router on (X, y) with the
// router's own standardisation (for checks against an independent backprop).
int tg_router_loss_grad(const tg_router *r, int n, const float *X, const float *y, float q, float *loss, float *grad)
{
    if (!r || n < 1 || !X || !y || !loss || !grad || !(q > 0.f && q < 1.f)) return TG_EINVAL;
    DevBufs B;
    float *dX, *dy, *dmu, *dsd, *dp, *dg, *dl, *gpart, *lpart;
    const int nblk = (n + TRB - 1) / TRB;
    TG_CUDA(B.alloc(&dX, (size_t)n * NFEAT));
    TG_CUDA(B.alloc(&dy, n));
    TG_CUDA(B.alloc(&dmu, NFEAT));
    TG_CUDA(B.alloc(&dsd, NFEAT));
    TG_CUDA(B.alloc(&dp, NPARAM));
    TG_CUDA(B.alloc(&dg, NPARAM));
    TG_CUDA(B.alloc(&dl, 1));
    TG_CUDA(B.alloc(&gpart, (size_t)nblk * NPARAM));
    TG_CUDA(B.alloc(&lpart, nblk));
    TG_CUDA(cudaMemcpy(dX, X, sizeof(float) * n * NFEAT, cudaMemcpyHostToDevice));
    TG_CUDA(cudaMemcpy(dy, y, sizeof(float) * n, cudaMemcpyHostToDevice));
    TG_CUDA(cudaMemcpy(dmu, r->mu, sizeof(float) * NFEAT, cudaMemcpyHostToDevice));
    TG_CUDA(cudaMemcpy(dsd, r->sd, sizeof(float) * NFEAT, cudaMemcpyHostToDevice));
    TG_CUDA(cudaMemcpy(dp, r->params, sizeof(float) * NPARAM, cudaMemcpyHostToDevice));
    int rc = router_loss_grad_dev(r, n, dX, dy, dmu, dsd, dp, q, dg, dl, gpart, lpart);
    if (rc != TG_OK) return rc;
    TG_CUDA(cudaMemcpy(grad, dg, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost));
    TG_CUDA(cudaMemcpy(loss, dl, sizeof(float), cudaMemcpyDeviceToHost));
    return TG_OK;
}

int tg_router_predict(const tg_router *r, int n, const float *X, float *out)
{
    if (!r || n < 1 || !X || !out) return TG_EINVAL;
    DevBufs B;
    float *dX, *dmu, *dsd, *dp, *dout;
    TG_CUDA(B.alloc(&dX, (size_t)n * NFEAT));
    TG_CUDA(B.alloc(&dmu, NFEAT));
    TG_CUDA(B.alloc(&dsd, NFEAT));
    TG_CUDA(B.alloc(&dp, NPARAM));
    TG_CUDA(B.alloc(&dout, n));
    TG_CUDA(cudaMemcpy(dX, X, sizeof(float) * n * NFEAT, cudaMemcpyHostToDevice));
    TG_CUDA(cudaMemcpy(dmu, r->mu, sizeof(float) * NFEAT, cudaMemcpyHostToDevice));
    TG_CUDA(cudaMemcpy(dsd, r->sd, sizeof(float) * NFEAT, cudaMemcpyHostToDevice));
    TG_CUDA(cudaMemcpy(dp, r->params, sizeof(float) * NPARAM, cudaMemcpyHostToDevice));
    k_mlp_predict<<<(n + 127) / 128, 128>>>(n, dX, dmu, dsd, dp, dout);
    TG_CUDA(cudaGetLastError());
    TG_CUDA(cudaMemcpy(out, dout, sizeof(float) * n, cudaMemcpyDeviceToHost));
    return TG_OK;
}

// File: "TGRT", version 1, NFEAT, NH, then params, mu, sd, margin, eps_rel, trained.
int tg_router_save(const tg_router *r, const char *path)
{
    if (!r || !path) return TG_EINVAL;
    FILE *f = std::fopen(path, "wb");
    if (!f) return TG_EINVAL;
    const int hdr[4] = {0x54524754, 1, NFEAT, NH};
    bool ok = std::fwrite(hdr, sizeof(hdr), 1, f) == 1 && std::fwrite(r->params, sizeof(r->params), 1, f) == 1 &&
              std::fwrite(r->mu, sizeof(r->mu), 1, f) == 1 && std::fwrite(r->sd, sizeof(r->sd), 1, f) == 1;
    const float cal[3] = {r->margin, r->eps_rel, (float)r->trained};
    ok = ok && std::fwrite(cal, sizeof(cal), 1, f) == 1;
    ok = (std::fclose(f) == 0) && ok;
    return ok ? TG_OK : TG_EINVAL;
}

int tg_router_load(const char *path, tg_router **out)
{
    if (!path || !out) return TG_EINVAL;
    *out = nullptr;
    FILE *f = std::fopen(path, "rb");
    if (!f) return TG_EROUTER;
    int hdr[4];
    tg_router *r = new (std::nothrow) tg_router();
    float cal[3];
    bool ok = r && std::fread(hdr, sizeof(hdr), 1, f) == 1 && hdr[0] == 0x54524754 && hdr[1] == 1 &&
              hdr[2] == NFEAT && hdr[3] == NH && std::fread(r->params, sizeof(r->params), 1, f) == 1 &&
              std::fread(r->mu, sizeof(r->mu), 1, f) == 1 && std::fread(r->sd, sizeof(r->sd), 1, f) == 1 &&
              std::fread(cal, sizeof(cal), 1, f) == 1;
    std::fclose(f);
    for (int k = 0; ok && k < NPARAM; ++k) ok = std::isfinite(r->params[k]);
    for (int j = 0; ok && j < NFEAT; ++j) ok = std::isfinite(r->mu[j]) && r->sd[j] > 0.f && std::isfinite(r->sd[j]);
    ok = ok && std::isfinite(cal[0]) && cal[1] >= 0.f && std::isfinite(cal[1]);
    if (!ok) {
        delete r;
        return TG_EROUTER;
    }
    r->margin = cal[0];
    r->eps_rel = cal[1];
    r->trained = cal[2] != 0.f;
    *out = r;
    return TG_OK;
}

}  // extern "C"
