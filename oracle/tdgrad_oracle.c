/*
 * CPU ORACLE for the two-electron term of the TDA-TDDFT nuclear gradient.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check and the benchmark's
 * CPU-baseline leg may load this library.  It shares no code, header, table or
 * constant generator with the CUDA path, and the CUDA path never calls it.
 *
 * What it computes (plain definition, fp64; Boys function in long double):
 *
 *   g[E,x] = sum_pairs sum_{mu nu lam sig, all ordered}
 *              [ c_J  d(mu nu|lam sig)/dE_x      A_{mu nu}  B_{lam sig}
 *              + c_K  d(mu nu|lam sig)/dE_x      A_{mu lam} B_{nu sig}
 *              + c_Klr d(mu nu|lam sig)_w/dE_x   A_{mu lam} B_{nu sig} ]
 *
 * i.e. the 4th and 5th terms of the AO gradient (Sec. II.A, eq. dE_ao) with
 * the two-particle densities Gamma, Gamma^lr of eq. gamma written as a list of
 * (A, B, c_J, c_K, c_K_lr, omega) pairs.  (|)_w is the erf(omega r)/r
 * operator of eq. lreri_k.
 *
 *  - Basis (Sec. II.C, eq. cartG): Cartesian Gaussians, components of a shell
 *    in lexicographic order (xx, xy, xz, yy, yz, zz); every component carries
 *    the x^l normalisation N_k N_c of its shell.
 *  - Primitive ERIs: Obara-Saika vertical recursion from [00|00]^(m) (Head-
 *    Gordon-Pople form), then the horizontal transfer written out as the
 *    binomial expansion (x-B_x)^b = sum_k C(b,k) (x-A_x)^k (A_x-B_x)^(b-k).
 *    The erf operator uses [00|00]^(m) = pref * theta^(2m+1) F_m(theta^2 T),
 *    theta^2 = w^2/(w^2+rho); the recursion coefficients are unchanged.
 *    Every vector of the recursion (P - A, Q - C, P - Q, W - P, W - Q) is
 *    formed from differences of centres, since the integrals depend on the
 *    relative positions only; the gradient is then invariant under a rigid
 *    shift of the molecule to rounding.
 *  - Derivatives (eqs. deriv, deri, eriupdate): d/dA_x of a primitive is
 *    2 zeta (l_x+1 term) - l_x (l_x-1 term).  ALL FOUR centres are
 *    differentiated explicitly; translational invariance is not used, so it
 *    is a test of this code.
 *  - Contraction: "plain" mode loops over every ordered shell quartet;
 *    "canonical" mode loops a>=b, c>=d, ab>=cd and applies the sum over the
 *    8 permutation images divided by the stabiliser size.
 *  - Screening (Sec. II.E: density-multiplied Schwarz bound, threshold tau):
 *    a canonical quartet is skipped iff bound_q < tau with
 *      bound_q = 8 * npair * max(Q'_ab Q_cd, Q_ab Q'_cd) * M_q^2,
 *      Q_ab  = max_{mu nu} sum_{kl} |c_k c_l| sqrt((k_mu l_nu|k_mu l_nu)),
 *      Q'_ab = same with the primitive mu (or nu) replaced by its derivative
 *              function along x, y or z, maximised over centre and direction,
 *      M(x,y)= max_p sqrt(|c_J|+|c_K|+|c_K_lr|) max(|A_p|,|B_p|) over the
 *              shell blocks (x,y) and (y,x),
 *      M_q   = max of M over the blocks ab, cd, ac, ad, bc, bd.
 *    With tau > 0 a primitive pair (k,l) of a shell pair is also dropped iff
 *      8 * npair * b_kl * max(Qmax, Q'max) * Mmax^2 < 1e-6 tau,
 *      b_kl = max over mu nu and over the plain and derivative charges of
 *             |c_k c_l| sqrt(self-repulsion) (the terms summed in Q and Q'),
 *    with Qmax, Q'max, Mmax the largest Q, Q', M of the system.
 *    tau = 0 keeps every quartet and primitive (no approximation at all).
 *  - Shards: a quartet belongs to shard (rank, nranks) iff
 *      max(key(a,b), key(c,d)) mod nranks == rank,
 *      key(x,y) = X(X+1)/2 + Y with X = max(x,y), Y = min(x,y).
 */
/* OR_MUTATION (default 0) plants one deliberate mistake for the mutation
 * test (tests/test_oracle_mutations.py), which builds the variants into a
 * temporary directory and checks that the pins catch each of them; the
 * oracle itself is always built with OR_MUTATION = 0. */
#ifndef OR_MUTATION
#define OR_MUTATION 0
#endif
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <stdint.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MAXL 2
#define OR_MAXT 5                 /* highest total angular momentum in tables */
#define OR_NTRI 56                /* triples with total <= 5 */
#define OR_MMAX 12

/* ---------------------------------------------------------------- triples */
static int tri_x[OR_NTRI], tri_y[OR_NTRI], tri_z[OR_NTRI], tri_l[OR_NTRI];
static int tri_start[OR_MAXT + 2];
static int tri_idx[OR_MAXT + 1][OR_MAXT + 1][OR_MAXT + 1];
static int tri_ready = 0;

static void init_tri(void)
{
    if (tri_ready) return;
    int n = 0;
    for (int L = 0; L <= OR_MAXT; ++L) {
        tri_start[L] = n;
        for (int lx = L; lx >= 0; --lx)
            for (int ly = L - lx; ly >= 0; --ly) {
                int lz = L - lx - ly;
                tri_x[n] = lx; tri_y[n] = ly; tri_z[n] = lz; tri_l[n] = L;
                tri_idx[lx][ly][lz] = n;
                ++n;
            }
    }
    tri_start[OR_MAXT + 1] = n;
    tri_ready = 1;
}

static inline int tcomp(int t, int i) { return i == 0 ? tri_x[t] : (i == 1 ? tri_y[t] : tri_z[t]); }
static inline int tshift(int t, int i, int d)
{
    int x = tri_x[t] + (i == 0 ? d : 0), y = tri_y[t] + (i == 1 ? d : 0), z = tri_z[t] + (i == 2 ? d : 0);
    if (x < 0 || y < 0 || z < 0 || x + y + z > OR_MAXT) return -1;
    return tri_idx[x][y][z];
}
static inline int ncart(int l) { return (l + 1) * (l + 2) / 2; }

/* ------------------------------------------------------------------ Boys */
/* F_m(T) = int_0^1 t^(2m) exp(-T t^2) dt for m = 0..mmax.
 * T <= 40: series e^-T sum_k (2T)^k / ((2m+1)(2m+3)...(2m+2k+1)) for the top
 * order, then downward recursion F_{m-1} = (2T F_m + e^-T)/(2m-1).
 * T > 40: F_0 = sqrt(pi/T) erf(sqrt T)/2 and upward recursion
 * F_{m+1} = ((2m+1) F_m - e^-T) / (2T). */
static void boys_ld(int mmax, long double T, long double *F)
{
    if (T <= 40.0L) {
        long double term = 1.0L / (2 * mmax + 1), sum = term;
        for (int k = 1; k < 2000; ++k) {
            term *= 2.0L * T / (long double)(2 * mmax + 2 * k + 1);
            sum += term;
            if (term < sum * 1e-22L) break;
        }
        long double et = expl(-T);
        F[mmax] = et * sum;
#if OR_MUTATION == 4
        for (int m = mmax; m > 0; --m) F[m - 1] = (2.0L * T * F[m] - et) / (long double)(2 * m - 1);
#else
        for (int m = mmax; m > 0; --m) F[m - 1] = (2.0L * T * F[m] + et) / (long double)(2 * m - 1);
#endif
    } else {
        long double et = expl(-T);
        F[0] = 0.5L * sqrtl(3.14159265358979323846264338327950288L / T) * erfl(sqrtl(T));
#if OR_MUTATION == 12
        for (int m = 0; m < mmax; ++m) F[m + 1] = ((long double)(2 * m + 1) * F[m] + et) / (2.0L * T);
#else
        for (int m = 0; m < mmax; ++m) F[m + 1] = ((long double)(2 * m + 1) * F[m] - et) / (2.0L * T);
#endif
    }
}

/* branch selector exposed for the overlap-region pin: 0 = automatic,
 * 1 = series + downward, 2 = erf + upward */
void or_boys(int mmax, double T, int branch, double *out)
{
    long double F[64];
    long double t = T;
    if (mmax > 60) mmax = 60;
    if (branch == 1) {
        long double term = 1.0L / (2 * mmax + 1), sum = term;
        for (int k = 1; k < 20000; ++k) {
            term *= 2.0L * t / (long double)(2 * mmax + 2 * k + 1);
            sum += term;
            if (term < sum * 1e-22L) break;
        }
        long double et = expl(-t);
        F[mmax] = et * sum;
        for (int m = mmax; m > 0; --m) F[m - 1] = (2.0L * t * F[m] + et) / (long double)(2 * m - 1);
    } else if (branch == 2 && T > 0) {
        long double et = expl(-t);
        F[0] = 0.5L * sqrtl(3.14159265358979323846264338327950288L / t) * erfl(sqrtl(t));
        for (int m = 0; m < mmax; ++m) F[m + 1] = ((long double)(2 * m + 1) * F[m] - et) / (2.0L * t);
    } else {
        boys_ld(mmax, t, F);
    }
    for (int m = 0; m <= mmax; ++m) out[m] = (double)F[m];
}

/* ----------------------------------------------------------------- basis */
typedef struct {
    int natom, nshell, nbf;
    const double *xyz;
    const int *sh_atom, *sh_l, *sh_nprim;
    int *sh_off, *bf_off;
    const double *exps;
    double *cn;           /* d_k N_k N_c */
} obasis;

static double dfact(int n) { double r = 1.0; for (int k = n; k > 1; k -= 2) r *= k; return r; }

/* Normalised contraction coefficients (Sec. II.C eq. cartG, x^l convention):
 * N_k = (2 z/pi)^(3/4) (4 z)^(l/2) / sqrt((2l-1)!!),
 * N_c^-2 = sum_kk' d_k d_k' N_k N_k' (pi/(z_k+z_k'))^(3/2) (2l-1)!! / (2(z_k+z_k'))^l */
void or_normalise(int nshell, const int *sh_l, const int *sh_nprim, const double *exps,
                  const double *coefs, double *out)
{
    int off = 0;
    for (int s = 0; s < nshell; ++s) {
        int l = sh_l[s], K = sh_nprim[s];
        double df = dfact(2 * l - 1);
        double nk[64];
        for (int k = 0; k < K; ++k) {
            double z = exps[off + k];
#if OR_MUTATION == 5
            nk[k] = pow(2.0 * z / M_PI, 0.75) * pow(4.0 * z, 1.0 * l) / sqrt(df);
#else
            nk[k] = pow(2.0 * z / M_PI, 0.75) * pow(4.0 * z, 0.5 * l) / sqrt(df);
#endif
        }
        double s2 = 0.0;
        for (int k = 0; k < K; ++k)
            for (int j = 0; j < K; ++j) {
                double zz = exps[off + k] + exps[off + j];
                s2 += coefs[off + k] * coefs[off + j] * nk[k] * nk[j] * pow(M_PI / zz, 1.5) * df / pow(2.0 * zz, l);
            }
        double nc = 1.0 / sqrt(s2);
        for (int k = 0; k < K; ++k) out[off + k] = coefs[off + k] * nk[k] * nc;
        off += K;
    }
}

static void basis_setup(obasis *b, int natom, const double *xyz, int nshell, const int *sh_atom,
                        const int *sh_l, const int *sh_nprim, const double *exps, const double *coefs)
{
    b->natom = natom; b->nshell = nshell; b->xyz = xyz;
    b->sh_atom = sh_atom; b->sh_l = sh_l; b->sh_nprim = sh_nprim; b->exps = exps;
    b->sh_off = (int *)malloc(sizeof(int) * (nshell + 1));
    b->bf_off = (int *)malloc(sizeof(int) * (nshell + 1));
    int off = 0, bo = 0;
    for (int s = 0; s < nshell; ++s) { b->sh_off[s] = off; b->bf_off[s] = bo; off += sh_nprim[s]; bo += ncart(sh_l[s]); }
    b->sh_off[nshell] = off; b->bf_off[nshell] = bo; b->nbf = bo;
    b->cn = (double *)malloc(sizeof(double) * (off > 0 ? off : 1));
    or_normalise(nshell, sh_l, sh_nprim, exps, coefs, b->cn);
}

static void basis_free(obasis *b) { free(b->sh_off); free(b->bf_off); free(b->cn); }

/* --------------------------------------------------- primitive VRR tables */
typedef struct {
    double *V;        /* [OR_NTRI][OR_NTRI][OR_MMAX] */
} vrr_ws;

#define VIX(e, f, m) (((size_t)(e) * OR_NTRI + (f)) * OR_MMAX + (m))

/* [e0|f0]^(0..) for |e| <= Le, |f| <= Lf for one primitive quartet, with e
 * on A (or on B when bra_on_b) and f on C (or on D when ket_on_d); the other
 * centre of each pair carries an s function.
 * omega <= 0: Coulomb 1/r; omega > 0: erf(omega r)/r (omega = inf allowed). */
static void vrr(vrr_ws *w, int Le, int Lf,
                double za, const double *A, double zb, const double *B,
                double zc, const double *C, double zd, const double *D, double omega,
                int bra_on_b, int ket_on_d)
{
    double p = za + zb, q = zc + zd;
    double PA[3], WP[3], QC[3], WQ[3];
    double ab2 = 0, cd2 = 0, pq2 = 0;
    /* The integrals depend on relative positions only: P - A = zb/p (B - A),
       P - B = za/p (A - B), the same for Q, and P - Q = (A - C) + (P - A) -
       (Q - C), W - P = q/(p+q) (Q - P), W - Q = p/(p+q) (P - Q), all from
       centre differences (no difference of absolute positions near each
       other, which would lose digits away from the origin). */
    for (int i = 0; i < 3; ++i) {
        const double ab = A[i] - B[i], cd = C[i] - D[i];
        ab2 += ab * ab;
        cd2 += cd * cd;
#if OR_MUTATION == 16
        /* product centres as absolute positions, differences taken afterwards */
        const double Pi = (za * A[i] + zb * B[i]) / p, Qi = (zc * C[i] + zd * D[i]) / q;
        const double pa = Pi - A[i], pb = Pi - B[i], qc = Qi - C[i], qd = Qi - D[i];
        const double pq = Pi - Qi;
#else
        const double pa = -zb / p * ab, pb = za / p * ab, qc = -zd / q * cd, qd = zc / q * cd;
        const double pq = (A[i] - C[i]) + pa - qc;
#endif
        pq2 += pq * pq;
        PA[i] = bra_on_b ? pb : pa;
        QC[i] = ket_on_d ? qd : qc;
        WP[i] = -q / (p + q) * pq;
        WQ[i] = p / (p + q) * pq;
    }
    double rho = p * q / (p + q);
    double T = rho * pq2;
    int M = Le + Lf;
    double pref = 2.0 * pow(M_PI, 2.5) / (p * q * sqrt(p + q)) * exp(-za * zb / p * ab2) * exp(-zc * zd / q * cd2);
    long double F[OR_MMAX + 2];
    double G[OR_MMAX + 2];
    if (omega > 0) {
        double th2 = isinf(omega) ? 1.0 : omega * omega / (omega * omega + rho);
        boys_ld(M, (long double)th2 * (long double)T, F);
#if OR_MUTATION == 3
        double thp = 1.0;
#else
        double th = sqrt(th2), thp = th;
#endif
        for (int m = 0; m <= M; ++m) { G[m] = (double)F[m] * thp; thp *= th2; }
    } else {
        boys_ld(M, (long double)T, F);
        for (int m = 0; m <= M; ++m) G[m] = (double)F[m];
    }
    double *V = w->V;
    for (int m = 0; m <= M; ++m) V[VIX(0, 0, m)] = pref * G[m];
    /* bra: [e0|00]^(m) */
    for (int e = 1; e < tri_start[Le + 1]; ++e) {
        int i = tri_x[e] > 0 ? 0 : (tri_y[e] > 0 ? 1 : 2);
        int em = tshift(e, i, -1);
        int emi = tcomp(em, i);
        int emm = emi > 0 ? tshift(em, i, -1) : -1;
        for (int m = 0; m <= M - tri_l[e]; ++m) {
            double v = PA[i] * V[VIX(em, 0, m)] + WP[i] * V[VIX(em, 0, m + 1)];
            if (emm >= 0) v += emi / (2.0 * p) * (V[VIX(emm, 0, m)] - rho / p * V[VIX(emm, 0, m + 1)]);
            V[VIX(e, 0, m)] = v;
        }
    }
    /* ket: [e0|f0]^(m) */
    for (int f = 1; f < tri_start[Lf + 1]; ++f) {
        int i = tri_x[f] > 0 ? 0 : (tri_y[f] > 0 ? 1 : 2);
        int fm = tshift(f, i, -1);
        int fmi = tcomp(fm, i);
        int fmm = fmi > 0 ? tshift(fm, i, -1) : -1;
        for (int e = 0; e < tri_start[Le + 1]; ++e) {
            int ei = tcomp(e, i);
            int em = ei > 0 ? tshift(e, i, -1) : -1;
            for (int m = 0; m <= M - tri_l[e] - tri_l[f]; ++m) {
                double v = QC[i] * V[VIX(e, fm, m)] + WQ[i] * V[VIX(e, fm, m + 1)];
                if (fmm >= 0) v += fmi / (2.0 * q) * (V[VIX(e, fmm, m)] - rho / q * V[VIX(e, fmm, m + 1)]);
#if OR_MUTATION == 2
                if (em >= 0) v -= ei / (2.0 * (p + q)) * V[VIX(em, fm, m + 1)];
#else
                if (em >= 0) v += ei / (2.0 * (p + q)) * V[VIX(em, fm, m + 1)];
#endif
                V[VIX(e, f, m)] = v;
            }
        }
    }
}

/* ------------------------------------------------ binomial transfer (HRR) */
static double binom(int n, int k)
{
    static const double c[4][4] = {{1, 0, 0, 0}, {1, 1, 0, 0}, {1, 2, 1, 0}, {1, 3, 3, 1}};
    return c[n][k];
}

/* (a b|c d) from a table T[e][f] = [e0|f0]^(0).  Orientation bit 1 (bra)
 * says e sits on B instead of A; bit 2 (ket) says f sits on D instead of C.
 * The angular factor on the other centre is expanded around the built one:
 * (x-B_x)^b = sum_k C(b,k) (x-A_x)^k (A_x-B_x)^(b-k)  (and A<->B, C<->D). */
static double hrr(const double *Tab, int orient, int a, int b, int c, int d, const double *AB, const double *CD)
{
    int bo = orient & 1, ko = (orient >> 1) & 1;
    int e0 = bo ? b : a, x = bo ? a : b;       /* built index, expanded index */
    int f0 = ko ? d : c, y = ko ? c : d;
#if OR_MUTATION == 9
    double sb = bo ? 1.0 : -1.0, sk = ko ? -1.0 : 1.0;
#else
    double sb = bo ? -1.0 : 1.0, sk = ko ? -1.0 : 1.0;   /* (B-A) = -(A-B) */
#endif
    double R1[3] = {sb * AB[0], sb * AB[1], sb * AB[2]}, R2[3] = {sk * CD[0], sk * CD[1], sk * CD[2]};
    int ex = tri_x[e0], ey = tri_y[e0], ez = tri_z[e0];
    int xx = tri_x[x], xy = tri_y[x], xz = tri_z[x];
    int fx = tri_x[f0], fy = tri_y[f0], fz = tri_z[f0];
    int yx = tri_x[y], yy = tri_y[y], yz = tri_z[y];
    double sum = 0.0;
    for (int kx = 0; kx <= xx; ++kx)
        for (int ky = 0; ky <= xy; ++ky)
            for (int kz = 0; kz <= xz; ++kz) {
                double wb = binom(xx, kx) * binom(xy, ky) * binom(xz, kz) *
                            pow(R1[0], xx - kx) * pow(R1[1], xy - ky) * pow(R1[2], xz - kz);
                int e = tri_idx[ex + kx][ey + ky][ez + kz];
                for (int jx = 0; jx <= yx; ++jx)
                    for (int jy = 0; jy <= yy; ++jy)
                        for (int jz = 0; jz <= yz; ++jz) {
                            double wd = binom(yx, jx) * binom(yy, jy) * binom(yz, jz) *
                                        pow(R2[0], yx - jx) * pow(R2[1], yy - jy) * pow(R2[2], yz - jz);
                            int f = tri_idx[fx + jx][fy + jy][fz + jz];
                            sum += wb * wd * Tab[(size_t)e * OR_NTRI + f];
                        }
            }
    return sum;
}

/* -------------------------------------------- contracted shell quartet */
/* Weighted contracted tables per operator, per orientation (see hrr) and per
 * slot: slot 0 weight 1, slot 1+X weight 2 zeta_X (X = A, B, C, D).  Each is
 * [e][f] at m = 0.  A primitive quartet is built on the tighter centre of
 * each pair (ties: A, C), which keeps the transfer free of cancellation. */
typedef struct {
    vrr_ws w;
    double *T[2][4][5];   /* [op][orient][slot] */
    int used[2][4];
} quartet_ws;

static void ws_alloc(quartet_ws *q)
{
    q->w.V = (double *)malloc(sizeof(double) * OR_NTRI * OR_NTRI * OR_MMAX);
    for (int o = 0; o < 2; ++o)
        for (int r = 0; r < 4; ++r)
            for (int s = 0; s < 5; ++s) q->T[o][r][s] = (double *)malloc(sizeof(double) * OR_NTRI * OR_NTRI);
}
static void ws_free(quartet_ws *q)
{
    free(q->w.V);
    for (int o = 0; o < 2; ++o)
        for (int r = 0; r < 4; ++r)
            for (int s = 0; s < 5; ++s) free(q->T[o][r][s]);
}

/* Contract the primitive tables of shells (a,b,c,d) for operator list ops
 * (op 0 = Coulomb; op 1 = erf with omega) into q->T.  deriv selects whether
 * the extents include the +1 needed by derivatives and the 2 zeta weights. */
static void contract_tables(const obasis *bs, quartet_ws *q, int sa, int sb, int sc, int sd,
                            int nops, const double *omegas, int deriv, const unsigned char *keep_ab,
                            const unsigned char *keep_cd)
{
    int la = bs->sh_l[sa], lb = bs->sh_l[sb], lc = bs->sh_l[sc], ld = bs->sh_l[sd];
    int Le = la + lb + deriv, Lf = lc + ld + deriv;
    int ne = tri_start[Le + 1], nf = tri_start[Lf + 1];
    const double *A = bs->xyz + 3 * bs->sh_atom[sa], *B = bs->xyz + 3 * bs->sh_atom[sb];
    const double *C = bs->xyz + 3 * bs->sh_atom[sc], *D = bs->xyz + 3 * bs->sh_atom[sd];
    int nslot = deriv ? 5 : 1;
    for (int o = 0; o < nops; ++o)
        for (int r = 0; r < 4; ++r) {
            q->used[o][r] = 0;
            for (int s = 0; s < nslot; ++s)
                for (int e = 0; e < ne; ++e)
                    for (int f = 0; f < nf; ++f) q->T[o][r][s][e * OR_NTRI + f] = 0.0;
        }
    for (int ka = 0; ka < bs->sh_nprim[sa]; ++ka)
        for (int kb = 0; kb < bs->sh_nprim[sb]; ++kb)
            for (int kc = 0; kc < bs->sh_nprim[sc]; ++kc)
                for (int kd = 0; kd < bs->sh_nprim[sd]; ++kd) {
                    if (keep_ab && !keep_ab[ka * bs->sh_nprim[sb] + kb]) continue;
                    if (keep_cd && !keep_cd[kc * bs->sh_nprim[sd] + kd]) continue;
                    double za = bs->exps[bs->sh_off[sa] + ka], zb = bs->exps[bs->sh_off[sb] + kb];
                    double zc = bs->exps[bs->sh_off[sc] + kc], zd = bs->exps[bs->sh_off[sd] + kd];
#if OR_MUTATION == 13
                    double cc = bs->cn[bs->sh_off[sa] + ka] * bs->cn[bs->sh_off[sb] + kb] *
                                bs->cn[bs->sh_off[sc] + kc] * bs->cn[bs->sh_off[sd] + kc % bs->sh_nprim[sd]];
#elif OR_MUTATION == 14
                    double cc = bs->cn[bs->sh_off[sa] + ka] * bs->cn[bs->sh_off[sb]] *
                                bs->cn[bs->sh_off[sc] + kc] * bs->cn[bs->sh_off[sd] + kd];
#else
                    double cc = bs->cn[bs->sh_off[sa] + ka] * bs->cn[bs->sh_off[sb] + kb] *
                                bs->cn[bs->sh_off[sc] + kc] * bs->cn[bs->sh_off[sd] + kd];
#endif
                    double wts[5] = {cc, cc * 2 * za, cc * 2 * zb, cc * 2 * zc, cc * 2 * zd};
                    int bo = zb > za, ko = zd > zc, r = bo | (ko << 1);
                    for (int o = 0; o < nops; ++o) {
                        vrr(&q->w, Le, Lf, za, A, zb, B, zc, C, zd, D, omegas[o], bo, ko);
                        q->used[o][r] = 1;
                        for (int s = 0; s < nslot; ++s) {
                            double *T = q->T[o][r][s];
                            for (int e = 0; e < ne; ++e)
                                for (int f = 0; f < nf; ++f) T[e * OR_NTRI + f] += wts[s] * q->w.V[VIX(e, f, 0)];
                        }
                    }
                }
}

/* contracted (a b|c d) of operator o from weighted slot s */
static double tab_int(const quartet_ws *q, int o, int s, int a, int b, int c, int d,
                      const double *AB, const double *CD)
{
    double v = 0.0;
    for (int r = 0; r < 4; ++r)
        if (q->used[o][r]) v += hrr(q->T[o][r][s], r, a, b, c, d, AB, CD);
    return v;
}

/* derivative of (a b|c d) w.r.t. centre X (0..3) along direction i, operator
 * o: 2 zeta (X+1_i) - X_i (X-1_i). */
static double deriv_int(const quartet_ws *q, int o, int X, int i, int a, int b, int c, int d,
                        const double *AB, const double *CD)
{
    int t[4] = {a, b, c, d};
    int ni = tcomp(t[X], i);
    int tu[4] = {a, b, c, d};
    tu[X] = tshift(t[X], i, +1);
    double v = tab_int(q, o, 1 + X, tu[0], tu[1], tu[2], tu[3], AB, CD);
    if (ni > 0 && OR_MUTATION != 1) {
        int td[4] = {a, b, c, d};
        td[X] = tshift(t[X], i, -1);
        v -= ni * tab_int(q, o, 0, td[0], td[1], td[2], td[3], AB, CD);
    }
    return v;
}

/* -------------------------------------------------------- public helpers */
/* Contracted integrals (ab|cd) of one shell quartet, all components, for one
 * operator (omega <= 0: 1/r; omega > 0: erf(omega r)/r).  out[na][nb][nc][nd]. */
void or_shell_eri(int natom, const double *xyz, int nshell, const int *sh_atom, const int *sh_l,
                  const int *sh_nprim, const double *exps, const double *coefs,
                  int sa, int sb, int sc, int sd, double omega, double *out)
{
    init_tri();
    obasis bs;
    basis_setup(&bs, natom, xyz, nshell, sh_atom, sh_l, sh_nprim, exps, coefs);
    quartet_ws q;
    ws_alloc(&q);
    double om[1] = {omega};
    contract_tables(&bs, &q, sa, sb, sc, sd, 1, om, 0, NULL, NULL);
    const double *A = xyz + 3 * sh_atom[sa], *B = xyz + 3 * sh_atom[sb];
    const double *C = xyz + 3 * sh_atom[sc], *D = xyz + 3 * sh_atom[sd];
    double AB[3] = {A[0] - B[0], A[1] - B[1], A[2] - B[2]}, CD[3] = {C[0] - D[0], C[1] - D[1], C[2] - D[2]};
    int la = sh_l[sa], lb = sh_l[sb], lc = sh_l[sc], ld = sh_l[sd];
    int n = 0;
    for (int i = 0; i < ncart(la); ++i)
        for (int j = 0; j < ncart(lb); ++j)
            for (int k = 0; k < ncart(lc); ++k)
                for (int l = 0; l < ncart(ld); ++l)
                    out[n++] = tab_int(&q, 0, 0, tri_start[la] + i, tri_start[lb] + j, tri_start[lc] + k,
                                       tri_start[ld] + l, AB, CD);
    ws_free(&q);
    basis_free(&bs);
}

/* Derivative integrals of one shell quartet: out[4 centres][3][na][nb][nc][nd]
 * = d(ab|cd)/dX_i, centres in the order a, b, c, d. */
void or_shell_eri_deriv(int natom, const double *xyz, int nshell, const int *sh_atom, const int *sh_l,
                        const int *sh_nprim, const double *exps, const double *coefs,
                        int sa, int sb, int sc, int sd, double omega, double *out)
{
    init_tri();
    obasis bs;
    basis_setup(&bs, natom, xyz, nshell, sh_atom, sh_l, sh_nprim, exps, coefs);
    quartet_ws q;
    ws_alloc(&q);
    double om[1] = {omega};
    contract_tables(&bs, &q, sa, sb, sc, sd, 1, om, 1, NULL, NULL);
    const double *A = xyz + 3 * sh_atom[sa], *B = xyz + 3 * sh_atom[sb];
    const double *C = xyz + 3 * sh_atom[sc], *D = xyz + 3 * sh_atom[sd];
    double AB[3] = {A[0] - B[0], A[1] - B[1], A[2] - B[2]}, CD[3] = {C[0] - D[0], C[1] - D[1], C[2] - D[2]};
    int la = sh_l[sa], lb = sh_l[sb], lc = sh_l[sc], ld = sh_l[sd];
    int na = ncart(la), nb = ncart(lb), nc = ncart(lc), nd = ncart(ld);
    size_t nq = (size_t)na * nb * nc * nd;
    for (int X = 0; X < 4; ++X)
        for (int i = 0; i < 3; ++i) {
            size_t n = 0;
            for (int a = 0; a < na; ++a)
                for (int b = 0; b < nb; ++b)
                    for (int c = 0; c < nc; ++c)
                        for (int d = 0; d < nd; ++d)
                            out[(X * 3 + i) * nq + n++] =
                                deriv_int(&q, 0, X, i, tri_start[la] + a, tri_start[lb] + b, tri_start[lc] + c,
                                          tri_start[ld] + d, AB, CD);
        }
    ws_free(&q);
    basis_free(&bs);
}

/* ------------------------------------------------------------- Schwarz */
/* Q_ab and Q'_ab (see header comment) from primitive self-repulsions. */
static void schwarz_pair(const obasis *bs, quartet_ws *q, int sa, int sb, double *Qo, double *Qdo, double *bprim)
{
    int la = bs->sh_l[sa], lb = bs->sh_l[sb];
    int na = ncart(la), nb = ncart(lb);
    const double *A = bs->xyz + 3 * bs->sh_atom[sa], *B = bs->xyz + 3 * bs->sh_atom[sb];
    double AB[3] = {A[0] - B[0], A[1] - B[1], A[2] - B[2]};
    double acc[36], accd[36 * 6];
    for (int n = 0; n < na * nb; ++n) acc[n] = 0.0;
    for (int n = 0; n < na * nb * 6; ++n) accd[n] = 0.0;
    int L = la + lb + 1;
    for (int ka = 0; ka < bs->sh_nprim[sa]; ++ka)
        for (int kb = 0; kb < bs->sh_nprim[sb]; ++kb) {
            double za = bs->exps[bs->sh_off[sa] + ka], zb = bs->exps[bs->sh_off[sb] + kb];
            double cc = fabs(bs->cn[bs->sh_off[sa] + ka] * bs->cn[bs->sh_off[sb] + kb]);
            int bo = zb > za, r = bo | (bo << 1);
            vrr(&q->w, L, L, za, A, zb, B, za, A, zb, B, 0.0, bo, bo);
            double *T = q->T[0][0][0];
            for (int e = 0; e < tri_start[L + 1]; ++e)
                for (int f = 0; f < tri_start[L + 1]; ++f) T[e * OR_NTRI + f] = q->w.V[VIX(e, f, 0)];
            double bmax = 0.0;
            for (int a = 0; a < na; ++a)
                for (int b = 0; b < nb; ++b) {
                    int ta = tri_start[la] + a, tb = tri_start[lb] + b;
                    double s = hrr(T, r, ta, tb, ta, tb, AB, AB);
                    acc[a * nb + b] += cc * sqrt(s > 0 ? s : 0.0);
                    if (cc * sqrt(s > 0 ? s : 0.0) > bmax) bmax = cc * sqrt(s > 0 ? s : 0.0);
                    for (int X = 0; X < 2; ++X)
                        for (int i = 0; i < 3; ++i) {
                            /* derivative function on centre X: 2z (+1_i) - n (-1_i) */
                            int t0 = X == 0 ? ta : tb;
                            int n = tcomp(t0, i);
                            double z = X == 0 ? za : zb;
                            int tp = tshift(t0, i, +1), tm = n > 0 ? tshift(t0, i, -1) : -1;
                            int tt[2] = {tp, tm};
                            double cf[2] = {2.0 * z, -(double)n};
                            double v = 0.0;
                            for (int u = 0; u < 2; ++u)
                                for (int w = 0; w < 2; ++w) {
                                    if (tt[u] < 0 || tt[w] < 0) continue;
                                    int a1 = X == 0 ? tt[u] : ta, b1 = X == 0 ? tb : tt[u];
                                    int a2 = X == 0 ? tt[w] : ta, b2 = X == 0 ? tb : tt[w];
                                    v += cf[u] * cf[w] * hrr(T, r, a1, b1, a2, b2, AB, AB);
                                }
                            accd[(a * nb + b) * 6 + X * 3 + i] += cc * sqrt(v > 0 ? v : 0.0);
                            if (cc * sqrt(v > 0 ? v : 0.0) > bmax) bmax = cc * sqrt(v > 0 ? v : 0.0);
                        }
                }
            if (bprim) bprim[ka * bs->sh_nprim[sb] + kb] = bmax;
        }
    double Q = 0.0, Qd = 0.0;
    for (int n = 0; n < na * nb; ++n) if (acc[n] > Q) Q = acc[n];
    for (int n = 0; n < na * nb * 6; ++n) if (accd[n] > Qd) Qd = accd[n];
    *Qo = Q;
    *Qdo = Qd;
}

/* Q and Q' for every ordered shell pair: Q[a*nshell+b]. */
void or_schwarz(int natom, const double *xyz, int nshell, const int *sh_atom, const int *sh_l,
                const int *sh_nprim, const double *exps, const double *coefs, double *Q, double *Qd)
{
    init_tri();
    obasis bs;
    basis_setup(&bs, natom, xyz, nshell, sh_atom, sh_l, sh_nprim, exps, coefs);
#pragma omp parallel
    {
        quartet_ws q;
        ws_alloc(&q);
#pragma omp for schedule(dynamic, 4)
        for (int a = 0; a < nshell; ++a)
            for (int b = 0; b <= a; ++b) {
                double x, y;
                schwarz_pair(&bs, &q, a, b, &x, &y, NULL);
                Q[a * nshell + b] = Q[b * nshell + a] = x;
                Qd[a * nshell + b] = Qd[b * nshell + a] = y;
            }
        ws_free(&q);
    }
    basis_free(&bs);
}

/* ------------------------------------------------------------ gradient */
static inline int64_t pairkey(int x, int y)
{
    int X = x > y ? x : y, Y = x > y ? y : x;
    return (int64_t)X * (X + 1) / 2 + Y;
}

typedef struct {
    int npair;
    const double *const *A, *const *B;
    const double *cJ, *cK, *cKlr;
    double omega;     /* shared lr omega (<= 0: no lr term) */
    int use_lr;
} opairs;

/* Gamma for the full-range (g0) and lr (g1) operators of the ordered function
 * quartet (m n | l s), summed over the density pairs. */
static inline void gamma_ordered(const opairs *pp, int nbf, int m, int n, int l, int s, double *g0, double *g1)
{
    double a0 = 0.0, a1 = 0.0;
    for (int p = 0; p < pp->npair; ++p) {
        const double *A = pp->A[p], *B = pp->B[p];
        double j = A[(size_t)m * nbf + n] * B[(size_t)l * nbf + s];
#if OR_MUTATION == 10
        double k = A[(size_t)l * nbf + m] * B[(size_t)n * nbf + s];
#else
        double k = A[(size_t)m * nbf + l] * B[(size_t)n * nbf + s];
#endif
        a0 += pp->cJ[p] * j + pp->cK[p] * k;
        a1 += pp->cKlr[p] * k;
    }
    *g0 = a0;
    *g1 = a1;
}

/* Process one shell quartet (sa sb | sc sd): gamma from the given function
 * (ordered or 8-image) rule, derivative integrals, scatter to atoms. */
static void do_quartet(const obasis *bs, quartet_ws *q, const opairs *pp, int sa, int sb, int sc, int sd,
                       int canonical, double scale, double *grad, double *energy, int want_grad,
                       const unsigned char *keep_ab, const unsigned char *keep_cd)
{
    int la = bs->sh_l[sa], lb = bs->sh_l[sb], lc = bs->sh_l[sc], ld = bs->sh_l[sd];
    int na = ncart(la), nb = ncart(lb), nc = ncart(lc), nd = ncart(ld);
    int oa = bs->bf_off[sa], ob = bs->bf_off[sb], oc = bs->bf_off[sc], od = bs->bf_off[sd];
    int nbf = bs->nbf;
    int nops = pp->use_lr ? 2 : 1;
    double omegas[2] = {0.0, pp->omega};
    contract_tables(bs, q, sa, sb, sc, sd, nops, omegas, want_grad, keep_ab, keep_cd);
    const double *A = bs->xyz + 3 * bs->sh_atom[sa], *B = bs->xyz + 3 * bs->sh_atom[sb];
    const double *C = bs->xyz + 3 * bs->sh_atom[sc], *D = bs->xyz + 3 * bs->sh_atom[sd];
    double AB[3] = {A[0] - B[0], A[1] - B[1], A[2] - B[2]}, CD[3] = {C[0] - D[0], C[1] - D[1], C[2] - D[2]};
    int atoms[4] = {bs->sh_atom[sa], bs->sh_atom[sb], bs->sh_atom[sc], bs->sh_atom[sd]};
    double gl[12];
    for (int k = 0; k < 12; ++k) gl[k] = 0.0;
    double el = 0.0;
    for (int a = 0; a < na; ++a)
        for (int b = 0; b < nb; ++b)
            for (int c = 0; c < nc; ++c)
                for (int d = 0; d < nd; ++d) {
                    int m = oa + a, n = ob + b, l = oc + c, s = od + d;
                    double g0 = 0.0, g1 = 0.0;
                    if (!canonical) {
                        gamma_ordered(pp, nbf, m, n, l, s, &g0, &g1);
                    } else {
                        /* the 8 images of (m n|l s) */
#if OR_MUTATION == 6
                        int img[8][4] = {{m, n, l, s}, {n, m, l, s}, {m, n, s, l}, {n, m, s, l},
                                         {l, s, m, n}, {s, l, m, n}, {l, s, m, n}, {s, l, n, m}};
#else
                        int img[8][4] = {{m, n, l, s}, {n, m, l, s}, {m, n, s, l}, {n, m, s, l},
                                         {l, s, m, n}, {s, l, m, n}, {l, s, n, m}, {s, l, n, m}};
#endif
                        for (int t = 0; t < 8; ++t) {
                            double x0, x1;
                            gamma_ordered(pp, nbf, img[t][0], img[t][1], img[t][2], img[t][3], &x0, &x1);
                            g0 += x0;
                            g1 += x1;
                        }
                        g0 *= scale;
                        g1 *= scale;
                    }
                    if (g0 == 0.0 && g1 == 0.0) continue;
                    int ta = tri_start[la] + a, tb = tri_start[lb] + b, tc = tri_start[lc] + c, td = tri_start[ld] + d;
                    double gs[2] = {g0, g1};
                    for (int o = 0; o < nops; ++o) {
                        if (gs[o] == 0.0) continue;
                        if (energy) el += gs[o] * tab_int(q, o, 0, ta, tb, tc, td, AB, CD);
                        if (want_grad)
                            for (int X = 0; X < 4; ++X)
                                for (int i = 0; i < 3; ++i)
                                    gl[X * 3 + i] += gs[o] * deriv_int(q, o, X, i, ta, tb, tc, td, AB, CD);
                    }
                }
    if (want_grad)
        for (int X = 0; X < 4; ++X)
            for (int i = 0; i < 3; ++i) grad[atoms[(OR_MUTATION == 8 && X == 2) ? 3 : X] * 3 + i] += gl[X * 3 + i];
    if (energy) *energy += el;
}

/* Block max |.| of a matrix over shell blocks: out[x*nshell+y] over (x,y) and (y,x). */
static void block_max(const obasis *bs, const double *Mx, double *out)
{
    int ns = bs->nshell, nbf = bs->nbf;
    for (int x = 0; x < ns; ++x)
        for (int y = 0; y < ns; ++y) {
            double m = 0.0;
            for (int i = bs->bf_off[x]; i < bs->bf_off[x + 1]; ++i)
                for (int j = bs->bf_off[y]; j < bs->bf_off[y + 1]; ++j) {
                    double v1 = fabs(Mx[(size_t)i * nbf + j]), v2 = fabs(Mx[(size_t)j * nbf + i]);
                    if (v1 > m) m = v1;
                    if (v2 > m) m = v2;
                }
            out[x * ns + y] = m;
        }
}

/* Angular class of a shell quartet: with the pair class of a shell pair
 * P(x,y) = L(L+1)/2 + l, L = max(l_x,l_y), l = min(l_x,l_y) (ss ps pp ds dp dd
 * = 0..5), the quartet class is P1(P1+1)/2 + P2 with P1 >= P2 the larger and
 * smaller pair class of (ab) and (cd): the 21 classes of l <= 2 (Sec. II.C). */
static int quartet_class(const obasis *bs, int a, int b, int c, int d)
{
    int la = bs->sh_l[a], lb = bs->sh_l[b], lc = bs->sh_l[c], ld = bs->sh_l[d];
    int L1 = la > lb ? la : lb, l1 = la > lb ? lb : la, L2 = lc > ld ? lc : ld, l2 = lc > ld ? ld : lc;
    int P = L1 * (L1 + 1) / 2 + l1, Q = L2 * (L2 + 1) / 2 + l2;
    int hi = P > Q ? P : Q, lo = P > Q ? Q : P;
    return hi * (hi + 1) / 2 + lo;
}

/*
 * The gradient.  mode 0 = plain (all ordered shell quartets, no screening,
 * no shards), mode 1 = canonical (8-fold, optional screening and shards).
 * want_grad / want_energy select the outputs (grad natom*3 overwritten,
 * energy scalar).  nquart_out (nullable) receives the number of canonical
 * shell quartets evaluated.  qclass >= 0 keeps only the quartets of that
 * angular class (quartet_class below); -1 keeps all.  Returns 0, or -1 on
 * bad arguments.
 */
int or_grad2e(int natom, const double *xyz, int nshell, const int *sh_atom, const int *sh_l,
              const int *sh_nprim, const double *exps, const double *coefs,
              int npair, const double *const *Am, const double *const *Bm, const double *cJ,
              const double *cK, const double *cKlr, const double *omega,
              int mode, double tau, int rank, int nranks, int nthreads,
              int want_grad, double *grad, double *energy, long long *nquart_out, int qclass)
{
    init_tri();
    if (natom < 1 || nshell < 1 || npair < 0 || nranks < 1 || rank < 0 || rank >= nranks) return -1;
    for (int s = 0; s < nshell; ++s) if (sh_l[s] < 0 || sh_l[s] > OR_MAXL || sh_nprim[s] < 1) return -1;
    obasis bs;
    basis_setup(&bs, natom, xyz, nshell, sh_atom, sh_l, sh_nprim, exps, coefs);
    opairs pp = {npair, Am, Bm, cJ, cK, cKlr, 0.0, 0};
    for (int p = 0; p < npair; ++p)
        if (cKlr[p] != 0.0 && omega[p] > 0) {
            if (pp.use_lr && omega[p] != pp.omega) { basis_free(&bs); return -1; }
            pp.use_lr = 1;
            pp.omega = omega[p];
        }
    /* pairs whose lr coefficient is inert keep c_K_lr but never reach op 1 */
    double *cKlr_eff = (double *)malloc(sizeof(double) * (npair > 0 ? npair : 1));
    for (int p = 0; p < npair; ++p) cKlr_eff[p] = (omega[p] > 0) ? cKlr[p] : 0.0;
    pp.cKlr = cKlr_eff;

    int ns = nshell;
    double *Q = NULL, *Qd = NULL, *Mb = NULL;
    if (mode == 1 && tau > 0) {
        Q = (double *)malloc(sizeof(double) * ns * ns);
        Qd = (double *)malloc(sizeof(double) * ns * ns);
        Mb = (double *)calloc((size_t)ns * ns, sizeof(double));
        or_schwarz(natom, xyz, nshell, sh_atom, sh_l, sh_nprim, exps, coefs, Q, Qd);
        double *tmp = (double *)malloc(sizeof(double) * ns * ns);
        for (int p = 0; p < npair; ++p) {
            double w = sqrt(fabs(cJ[p]) + fabs(cK[p]) + fabs(cKlr_eff[p]));
            for (int which = 0; which < 2; ++which) {
                block_max(&bs, which == 0 ? Am[p] : Bm[p], tmp);
                for (int k = 0; k < ns * ns; ++k) { double v = w * tmp[k]; if (v > Mb[k]) Mb[k] = v; }
            }
        }
        free(tmp);
    }
    /* primitive-pair keep masks (tau > 0) */
    unsigned char *keep = NULL;
    long long *keep_off = NULL;
    if (mode == 1 && tau > 0) {
        long long npr = (long long)ns * (ns + 1) / 2;
        keep_off = (long long *)malloc(sizeof(long long) * (npr + 1));
        long long o = 0;
        for (int a = 0; a < ns; ++a)
            for (int b = 0; b <= a; ++b) {
                keep_off[(long long)a * (a + 1) / 2 + b] = o;
                o += (long long)sh_nprim[a] * sh_nprim[b];
            }
        keep_off[npr] = o;
        keep = (unsigned char *)malloc(o > 0 ? o : 1);
        double qmax = 0.0, qdmax = 0.0, mmax = 0.0;
        for (int k = 0; k < ns * ns; ++k) {
            if (Q[k] > qmax) qmax = Q[k];
            if (Qd[k] > qdmax) qdmax = Qd[k];
            if (Mb[k] > mmax) mmax = Mb[k];
        }
        double qq = qmax > qdmax ? qmax : qdmax;
        double eps_p = 1e-6 * tau;
#pragma omp parallel
        {
            quartet_ws qw;
            ws_alloc(&qw);
            double bp[256];
#pragma omp for schedule(dynamic, 4)
            for (int a = 0; a < ns; ++a)
                for (int b = 0; b <= a; ++b) {
                    double x, y;
                    schwarz_pair(&bs, &qw, a, b, &x, &y, bp);
                    long long o2 = keep_off[(long long)a * (a + 1) / 2 + b];
                    for (int k = 0; k < sh_nprim[a] * sh_nprim[b]; ++k)
                        keep[o2 + k] = (8.0 * npair * bp[k] * qq * mmax * mmax < eps_p) ? 0 : 1;
                }
            ws_free(&qw);
        }
    }

#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
    int nth = omp_get_max_threads();
#else
    int nth = 1;
#endif
    double *gacc = (double *)calloc((size_t)nth * natom * 3, sizeof(double));
    double *eacc = (double *)calloc((size_t)nth, sizeof(double));
    long long *cnt = (long long *)calloc((size_t)nth, sizeof(long long));
    double *Ep = energy ? eacc : NULL;

    if (mode == 0) {
#pragma omp parallel
        {
#ifdef _OPENMP
            int t = omp_get_thread_num();
#else
            int t = 0;
#endif
            quartet_ws q;
            ws_alloc(&q);
#pragma omp for schedule(dynamic, 1) collapse(2)
            for (int a = 0; a < ns; ++a)
                for (int b = 0; b < ns; ++b)
                    for (int c = 0; c < ns; ++c)
                        for (int d = 0; d < ns; ++d) {
                            if (qclass >= 0 && quartet_class(&bs, a, b, c, d) != qclass) continue;
                            do_quartet(&bs, &q, &pp, a, b, c, d, 0, 1.0, gacc + (size_t)t * natom * 3,
                                       Ep ? Ep + t : NULL, want_grad, NULL, NULL);
                            cnt[t]++;
                        }
            ws_free(&q);
        }
    } else {
        long long npairs_tot = (long long)ns * (ns + 1) / 2;
#pragma omp parallel
        {
#ifdef _OPENMP
            int t = omp_get_thread_num();
#else
            int t = 0;
#endif
            quartet_ws q;
            ws_alloc(&q);
#pragma omp for schedule(dynamic, 1)
            for (long long ab = 0; ab < npairs_tot; ++ab) {
                if (ab % nranks != rank) continue;
                int a = (int)((sqrt(8.0 * (double)ab + 1.0) - 1.0) / 2.0);
                while ((long long)a * (a + 1) / 2 > ab) --a;
                while ((long long)(a + 1) * (a + 2) / 2 <= ab) ++a;
                int b = (int)(ab - (long long)a * (a + 1) / 2);
                for (int c = 0; c <= a; ++c)
                    for (int d = 0; d <= c; ++d) {
                        long long cd = (long long)c * (c + 1) / 2 + d;
                        if (cd > ab) continue;
                        if (qclass >= 0 && quartet_class(&bs, a, b, c, d) != qclass) continue;
                        if (tau > 0) {
                            double S1 = Qd[a * ns + b] * Q[c * ns + d], S2 = Q[a * ns + b] * Qd[c * ns + d];
                            double S = S1 > S2 ? S1 : S2;
                            double Mq = Mb[a * ns + b];
                            int bl[5][2] = {{c, d}, {a, c}, {a, d}, {b, c}, {b, d}};
                            for (int k = 0; k < 5; ++k) { double v = Mb[bl[k][0] * ns + bl[k][1]]; if (v > Mq) Mq = v; }
                            double bound = 8.0 * npair * S * Mq * Mq;
                            if (bound < tau) continue;
                        }
                        double scale = 1.0;
                        if (a == b) scale *= 0.5;
                        if (c == d) scale *= 0.5;
                        if (ab == cd && OR_MUTATION != 7) scale *= 0.5;
                        do_quartet(&bs, &q, &pp, a, b, c, d, 1, scale, gacc + (size_t)t * natom * 3,
                                   Ep ? Ep + t : NULL, want_grad, keep ? keep + keep_off[ab] : NULL,
                                   keep ? keep + keep_off[cd] : NULL);
                        cnt[t]++;
                    }
            }
            ws_free(&q);
        }
    }
    if (want_grad)
        for (int k = 0; k < natom * 3; ++k) {
            double s = 0.0;
            for (int t = 0; t < nth; ++t) s += gacc[(size_t)t * natom * 3 + k];
            grad[k] = s;
        }
    if (energy) {
        double s = 0.0;
        for (int t = 0; t < nth; ++t) s += eacc[t];
        *energy = s;
    }
    if (nquart_out) {
        long long s = 0;
        for (int t = 0; t < nth; ++t) s += cnt[t];
        *nquart_out = s;
    }
    free(gacc); free(eacc); free(cnt); free(cKlr_eff);
    free(Q); free(Qd); free(Mb); free(keep); free(keep_off);
    basis_free(&bs);
    return 0;
}

/*
 * Fock-type matrices of a list of density matrices (Sec. II.B, the
 * two-electron part of eqs. G_2e and zfock; the XC kernel term is not part
 * of it):
 *   F[mu nu] = sum_p sum_{lam sig} B_p[lam sig] ( c_J (mu nu|lam sig)
 *              + c_K (mu lam|nu sig) + c_K_lr (mu lam|nu sig)_w ),
 * one nbf x nbf matrix F (overwritten), row-major.  Plain definition: every
 * ordered shell quartet (a b|c d) is evaluated once; its integrals
 * (m n|l s), m in a, n in b, l in c, s in d, enter the Coulomb block
 * F[m][n] with B[l][s] and the exchange block F[m][l] with B[n][s].  No
 * screening.  Returns 0, or -1 on bad arguments.
 */
int or_fock2e(int natom, const double *xyz, int nshell, const int *sh_atom, const int *sh_l,
              const int *sh_nprim, const double *exps, const double *coefs,
              int npair, const double *const *Bm, const double *cJ, const double *cK,
              const double *cKlr, const double *omega, int nthreads, double *F)
{
    init_tri();
    if (natom < 1 || nshell < 1 || npair < 0 || !F) return -1;
    for (int s = 0; s < nshell; ++s) if (sh_l[s] < 0 || sh_l[s] > OR_MAXL || sh_nprim[s] < 1) return -1;
    obasis bs;
    basis_setup(&bs, natom, xyz, nshell, sh_atom, sh_l, sh_nprim, exps, coefs);
    int use_lr = 0;
    double om = 0.0;
    for (int p = 0; p < npair; ++p)
        if (cKlr[p] != 0.0 && omega[p] > 0) {
            if (use_lr && omega[p] != om) { basis_free(&bs); return -1; }
            use_lr = 1;
            om = omega[p];
        }
    const int nbf = bs.nbf, ns = nshell, nops = use_lr ? 2 : 1;
    const double omegas[2] = {0.0, om};
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
    int nth = omp_get_max_threads();
#else
    int nth = 1;
    (void)nthreads;
#endif
    double *acc = (double *)calloc((size_t)nth * nbf * nbf, sizeof(double));
#pragma omp parallel
    {
#ifdef _OPENMP
        int t = omp_get_thread_num();
#else
        int t = 0;
#endif
        double *Ft = acc + (size_t)t * nbf * nbf;
        quartet_ws q;
        ws_alloc(&q);
#pragma omp for schedule(dynamic, 1) collapse(2)
        for (int a = 0; a < ns; ++a)
            for (int b = 0; b < ns; ++b)
                for (int c = 0; c < ns; ++c)
                    for (int d = 0; d < ns; ++d) {
                        contract_tables(&bs, &q, a, b, c, d, nops, omegas, 0, NULL, NULL);
                        const double *A = bs.xyz + 3 * bs.sh_atom[a], *Bc = bs.xyz + 3 * bs.sh_atom[b];
                        const double *C = bs.xyz + 3 * bs.sh_atom[c], *D = bs.xyz + 3 * bs.sh_atom[d];
                        double AB[3] = {A[0] - Bc[0], A[1] - Bc[1], A[2] - Bc[2]};
                        double CD[3] = {C[0] - D[0], C[1] - D[1], C[2] - D[2]};
                        int la = bs.sh_l[a], lb = bs.sh_l[b], lc = bs.sh_l[c], ld = bs.sh_l[d];
                        for (int i = 0; i < ncart(la); ++i)
                            for (int j = 0; j < ncart(lb); ++j)
                                for (int k = 0; k < ncart(lc); ++k)
                                    for (int l = 0; l < ncart(ld); ++l) {
                                        int m = bs.bf_off[a] + i, n = bs.bf_off[b] + j;
                                        int lam = bs.bf_off[c] + k, sig = bs.bf_off[d] + l;
                                        int ta = tri_start[la] + i, tb = tri_start[lb] + j;
                                        int tc = tri_start[lc] + k, td = tri_start[ld] + l;
                                        double e0 = tab_int(&q, 0, 0, ta, tb, tc, td, AB, CD);
                                        double e1 = nops > 1 ? tab_int(&q, 1, 0, ta, tb, tc, td, AB, CD) : 0.0;
                                        for (int p = 0; p < npair; ++p) {
                                            const double *Bp = Bm[p];
                                            double clr = omega[p] > 0 ? cKlr[p] : 0.0;
                                            Ft[(size_t)m * nbf + n] += cJ[p] * e0 * Bp[(size_t)lam * nbf + sig];
#if OR_MUTATION == 15
                                            Ft[(size_t)m * nbf + lam] += (cK[p] * e0 + clr * e1) * Bp[(size_t)sig * nbf + n];
#else
                                            Ft[(size_t)m * nbf + lam] += (cK[p] * e0 + clr * e1) * Bp[(size_t)n * nbf + sig];
#endif
                                        }
                                    }
                    }
        ws_free(&q);
    }
    for (size_t k = 0; k < (size_t)nbf * nbf; ++k) {
        double s = 0.0;
        for (int t = 0; t < nth; ++t) s += acc[(size_t)t * nbf * nbf + k];
        F[k] = s;
    }
    free(acc);
    basis_free(&bs);
    return 0;
}
