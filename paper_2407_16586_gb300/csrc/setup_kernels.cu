// Set-up kernels: Boys table, basis normalisation, Schwarz factors, density
// block maxima, primitive-pair records, density symmetrisation, and the final
// fixed-order reduction of per-CTA partial gradients.
#include "setup_kernels.cuh"

namespace tg {

// F_m(T0) at T0 = i h for m = 0..BOYS_M: the series
// F_M(T) = e^-T sum_k (2T)^k / ((2M+1)(2M+3)...(2M+2k+1)) for the top order,
// then downward recursion F_{m-1} = (2T F_m + e^-T)/(2m-1).
__global__ void k_boys_table(double *tab)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= BOYS_NG) return;
    const double T = i * BOYS_H;
    double term = 1.0 / (2 * BOYS_M + 1), sum = term;
    for (int k = 1; k < 400; ++k) {
        term *= 2.0 * T / (2 * BOYS_M + 2 * k + 1);
        sum += term;
        if (term < sum * 1e-18) break;
    }
    const double et = exp(-T);
    double f = et * sum;
    float *ftab = reinterpret_cast<float *>(tab + BOYS_TAB);
    tab[i * (BOYS_M + 1) + BOYS_M] = f;
    ftab[i * (BOYS_M + 1) + BOYS_M] = (float)f;
    for (int m = BOYS_M; m > 0; --m) {
        f = (2.0 * T * f + et) / (2 * m - 1);
        tab[i * (BOYS_M + 1) + m - 1] = f;
        ftab[i * (BOYS_M + 1) + m - 1] = (float)f;
    }
}

// Normalised contraction coefficients, x^l convention (Sec. II.C, eq. cartG):
// N_k = (2z/pi)^(3/4) (4z)^(l/2) / sqrt((2l-1)!!), and N_c from
// N_c^-2 = sum_kk' d_k d_k' N_k N_k' (pi/(z_k+z_k'))^(3/2) (2l-1)!! / (2(z_k+z_k'))^l.
__global__ void k_normalise(int nshell, const int *sh_l, const int *sh_nprim, const int *sh_poff,
                            const double *exps, const double *coefs, double *cn)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nshell) return;
    const int l = sh_l[s], K = sh_nprim[s], o = sh_poff[s];
    const double df = (l == 2) ? 3.0 : 1.0;  // (2l-1)!! for l <= 2
    double s2 = 0.0;
    for (int k = 0; k < K; ++k) {
        const double zk = exps[o + k];
        const double nk = pow(2.0 * zk / M_PI, 0.75) * pow(4.0 * zk, 0.5 * l) / sqrt(df);
        for (int j = 0; j < K; ++j) {
            const double zj = exps[o + j];
            const double nj = pow(2.0 * zj / M_PI, 0.75) * pow(4.0 * zj, 0.5 * l) / sqrt(df);
            const double zz = zk + zj;
            s2 += coefs[o + k] * coefs[o + j] * nk * nj * pow(M_PI / zz, 1.5) * df / pow(2.0 * zz, l);
        }
    }
    const double nc = 1.0 / sqrt(s2);
    for (int k = 0; k < K; ++k) {
        const double zk = exps[o + k];
        const double nk = pow(2.0 * zk / M_PI, 0.75) * pow(4.0 * zk, 0.5 * l) / sqrt(df);
        cn[o + k] = coefs[o + k] * nk * nc;
    }
}

// 1-D Hermite coefficients with runtime extents (i <= 3, j <= 3).
__device__ void etab_rt(double E[4][4][8], int I, int J, double PA, double PB, double oo2p)
{
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j)
            for (int t = 0; t < 8; ++t) E[i][j][t] = 0.0;
    E[0][0][0] = 1.0;
    for (int i = 0; i < I; ++i)
        for (int t = 0; t <= i + 1; ++t) {
            double v = 0.0;
            if (t <= i) v = PA * E[i][0][t];
            if (t >= 1) v += oo2p * E[i][0][t - 1];
            if (t + 1 <= i) v += (t + 1) * E[i][0][t + 1];
            E[i + 1][0][t] = v;
        }
    for (int j = 0; j < J; ++j)
        for (int i = 0; i <= I; ++i)
            for (int t = 0; t <= i + j + 1; ++t) {
                double v = 0.0;
                if (t <= i + j) v = PB * E[i][j][t];
                if (t >= 1) v += oo2p * E[i][j][t - 1];
                if (t + 1 <= i + j) v += (t + 1) * E[i][j][t + 1];
                E[i][j + 1][t] = v;
            }
}

__device__ __forceinline__ void cart_of(int l, int c, int &x, int &y, int &z)
{
    // lexicographic components: l=1 x y z; l=2 xx xy xz yy yz zz
    const int tx[3][6] = {{0, 0, 0, 0, 0, 0}, {1, 0, 0, 0, 0, 0}, {2, 1, 1, 0, 0, 0}};
    const int ty[3][6] = {{0, 0, 0, 0, 0, 0}, {0, 1, 0, 0, 0, 0}, {0, 1, 0, 2, 1, 0}};
    x = tx[l][c];
    y = ty[l][c];
    z = l - x - y;
}

// Coulomb self-repulsion of a Hermite distribution h at zero separation:
// pref * sum_{h1,h2} h1 h2 (-1)^{|h2|} R_{h1+h2}(0), where R_{2a,2b,2c}(0) =
// (2a-1)!!(2b-1)!!(2c-1)!! (-2 rho)^n / (2n+1), n = a+b+c, odd entries vanish.
__device__ double self_repulsion(const double *h, int Lh, double rho)
{
    double r0[12];  // (-2 rho)^n / (2n+1)
    double f = 1.0;
    for (int n = 0; n <= 2 * Lh && n < 12; ++n) {
        r0[n] = f / (2 * n + 1);
        f *= -2.0 * rho;
    }
    const double dfe[6] = {1.0, 1.0, 3.0, 15.0, 105.0, 945.0};  // (2a-1)!! for a = 0..5
    double sum = 0.0;
    for (int t1 = 0; t1 <= Lh; ++t1)
        for (int u1 = 0; u1 <= Lh - t1; ++u1)
            for (int v1 = 0; v1 <= Lh - t1 - u1; ++v1) {
                const double h1 = h[hidx(t1, u1, v1)];
                if (h1 == 0.0) continue;
                for (int t2 = t1 & 1; t2 <= Lh; t2 += 2)
                    for (int u2 = u1 & 1; u2 <= Lh - t2; u2 += 2)
                        for (int v2 = v1 & 1; v2 <= Lh - t2 - u2; v2 += 2) {
                            const int a = (t1 + t2) / 2, b = (u1 + u2) / 2, c = (v1 + v2) / 2;
                            const double R = dfe[a] * dfe[b] * dfe[c] * r0[a + b + c];
                            const double sg = ((t2 + u2 + v2) & 1) ? -1.0 : 1.0;
                            sum += h1 * h[hidx(t2, u2, v2)] * sg * R;
                        }
            }
    return sum;
}

// Schwarz factors of shell pairs (see tdgrad.h): Q from primitive
// self-repulsions of the product charges, Q' with the derivative function
// (eq. deriv) on either centre, maximised over centre and direction.
__global__ void k_schwarz(int npairs, const int2 *pairs, const double *xyz, const int *sh_atom, const int *sh_l,
                          const int *sh_nprim, const int *sh_poff, const double *exps, const double *cn, double *Q,
                          double *Qd, const long long *bpoff, double *bp)
{
    const int ip = blockIdx.x * blockDim.x + threadIdx.x;
    if (ip >= npairs) return;
    const int a = pairs[ip].x, b = pairs[ip].y;
    const int la = sh_l[a], lb = sh_l[b];
    const int na = ncart(la), nb = ncart(lb);
    const double *A = xyz + 3 * sh_atom[a], *B = xyz + 3 * sh_atom[b];
    const double AB2 = (A[0] - B[0]) * (A[0] - B[0]) + (A[1] - B[1]) * (A[1] - B[1]) + (A[2] - B[2]) * (A[2] - B[2]);
    double acc[36];
    for (int k = 0; k < 36; ++k) acc[k] = 0.0;
    double accdv[36][6];
    for (int k = 0; k < 36; ++k)
        for (int v = 0; v < 6; ++v) accdv[k][v] = 0.0;
    const int L = la + lb + 1;
    double E[3][4][4][8];
    double h[56];
    for (int ka = 0; ka < sh_nprim[a]; ++ka)
        for (int kb = 0; kb < sh_nprim[b]; ++kb) {
            const double za = exps[sh_poff[a] + ka], zb = exps[sh_poff[b] + kb];
            const double cc = fabs(cn[sh_poff[a] + ka] * cn[sh_poff[b] + kb]);
            const double p = za + zb;
            const double Kab = exp(-za * zb / p * AB2);
            const double pref = 34.986836655249725 / (p * p * sqrt(2.0 * p)) * Kab * Kab;
            for (int d = 0; d < 3; ++d) {
                const double P = (za * A[d] + zb * B[d]) / p;
                etab_rt(E[d], la + 1, lb + 1, P - A[d], P - B[d], 0.5 / p);
            }
            double bmax = 0.0;
            for (int ia = 0; ia < na; ++ia)
                for (int jb = 0; jb < nb; ++jb) {
                    int ax, ay, az, bx, by, bz;
                    cart_of(la, ia, ax, ay, az);
                    cart_of(lb, jb, bx, by, bz);
                    const int e[3][2] = {{ax, bx}, {ay, by}, {az, bz}};
                    for (int var = 0; var < 7; ++var) {
                        // var 0: plain; 1..3: d/dA x,y,z; 4..6: d/dB x,y,z
                        for (int k = 0; k < 56; ++k) h[k] = 0.0;
                        const int X = var == 0 ? -1 : (var - 1) / 3, dir = var == 0 ? -1 : (var - 1) % 3;
                        double c1[3][8];
                        int n1[3];
                        for (int d = 0; d < 3; ++d) {
                            const int i = e[d][0], j = e[d][1];
                            if (d == dir) {
                                const double z2 = 2.0 * (X == 0 ? za : zb);
                                n1[d] = i + j + 1;
                                for (int t = 0; t <= n1[d]; ++t) {
                                    double v;
                                    if (X == 0) v = z2 * E[d][i + 1][j][t] - (i > 0 ? i * E[d][i - 1][j][t] : 0.0);
                                    else v = z2 * E[d][i][j + 1][t] - (j > 0 ? j * E[d][i][j - 1][t] : 0.0);
                                    c1[d][t] = v;
                                }
                            } else {
                                n1[d] = i + j;
                                for (int t = 0; t <= n1[d]; ++t) c1[d][t] = E[d][i][j][t];
                            }
                        }
                        for (int t = 0; t <= n1[0]; ++t)
                            for (int u = 0; u <= n1[1]; ++u)
                                for (int v = 0; v <= n1[2]; ++v) h[hidx(t, u, v)] = c1[0][t] * c1[1][u] * c1[2][v];
                        const int Lh = n1[0] + n1[1] + n1[2];
                        double s = pref * self_repulsion(h, Lh < L ? Lh : L, p * 0.5);
                        s = sqrt(s > 0.0 ? s : 0.0) * cc;
                        if (var == 0) acc[ia * nb + jb] += s;
                        else accdv[ia * nb + jb][var - 1] += s;
                        bmax = fmax(bmax, s);
                    }
                }
            bp[bpoff[ip] + ka * sh_nprim[b] + kb] = bmax;
        }
    double q = 0.0, qd = 0.0;
    for (int k = 0; k < na * nb; ++k) {
        q = fmax(q, acc[k]);
        for (int v = 0; v < 6; ++v) qd = fmax(qd, accdv[k][v]);
    }
    Q[ip] = q;
    Qd[ip] = qd;
}

// M(x,y) = max_p w_p max(|A_p|, |B_p|) over shell blocks (x,y) and (y,x),
// w_p = sqrt(|c_J| + |c_K| + |c_K_lr|).  One thread per (x >= y).
__global__ void k_blockmax(int nshell, const int *sh_bf, const int *sh_l, DensArgs den, const double *w,
                           double *M, double *Mrow)
{
    const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long npr = (long long)nshell * (nshell + 1) / 2;
    if (id >= npr) return;
    int x = (int)((sqrt(8.0 * (double)id + 1.0) - 1.0) * 0.5);
    while ((long long)x * (x + 1) / 2 > id) --x;
    while ((long long)(x + 1) * (x + 2) / 2 <= id) ++x;
    const int y = (int)(id - (long long)x * (x + 1) / 2);
    const int nbf = den.nbf;
    const int fx = sh_bf[x], fy = sh_bf[y], nx = ncart(sh_l[x]), ny = ncart(sh_l[y]);
    double m = 0.0;
    for (int p = 0; p < den.npair; ++p) {
        double ma = 0.0, mb = 0.0;
        for (int i = 0; i < nx; ++i)
            for (int j = 0; j < ny; ++j) {
                const size_t r = fx + i, c = fy + j;
                ma = fmax(ma, fmax(fabs(den.A[p][r * nbf + c]), fabs(den.A[p][c * nbf + r])));
                mb = fmax(mb, fmax(fabs(den.B[p][r * nbf + c]), fabs(den.B[p][c * nbf + r])));
            }
        m = fmax(m, fmax(w[p] * ma, w[p] * mb));
    }
    M[(size_t)x * nshell + y] = m;
    M[(size_t)y * nshell + x] = m;
}

__global__ void k_rowmax(int nshell, const double *M, double *Mrow)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= nshell) return;
    double m = 0.0;
    for (int y = 0; y < nshell; ++y) m = fmax(m, M[(size_t)x * nshell + y]);
    Mrow[x] = m;
}

// Primitive pairs of each kept shell pair that survive the primitive screen
// (scale * b_kl * qq * Mmax^2 >= eps_p; every pair when eps_p <= 0).  b_kl
// is stored per canonical pair (larger shell index first).
__device__ __forceinline__ bool prim_keep(const double *bp, long long o, int ka, int kb, int Ka, int Kb, bool fwd,
                                          double scale, double qq, double mmax, double eps_p)
{
    if (!(eps_p > 0.0)) return true;
    const double b = bp[o + (fwd ? ka * Kb + kb : kb * Ka + ka)];
    return !(scale * b * qq * mmax * mmax < eps_p);
}

__global__ void k_prim_count(int npairs, const int *psa, const int *psb, const int *key, const int *sh_nprim,
                             const long long *bpoff, const double *bp, double scale, double qq, double mmax,
                             double eps_p, int *np_out)
{
    const int ip = blockIdx.x * blockDim.x + threadIdx.x;
    if (ip >= npairs) return;
    const int a = psa[ip], b = psb[ip];
    const int Ka = sh_nprim[a], Kb = sh_nprim[b];
    const long long o = bpoff[key[ip]];
    const bool fwd = a >= b;
    int n = 0;
    for (int ka = 0; ka < Ka; ++ka)
        for (int kb = 0; kb < Kb; ++kb)
            n += prim_keep(bp, o, ka, kb, Ka, Kb, fwd, scale, qq, mmax, eps_p) ? 1 : 0;
    np_out[ip] = n;
}

// Primitive-pair records: p, P, K = c_a c_b exp(-za zb/p |AB|^2), za.
__global__ void k_prim_pairs(int npairs, const int *psa, const int *psb, const int *poff, const int *key,
                             const double *xyz, const int *sh_atom, const int *sh_nprim, const int *sh_poff,
                             const double *exps, const double *cn, const long long *bpoff, const double *bp,
                             double scale, double qq, double mmax, double eps_p, double *p_, double *Px, double *Py,
                             double *Pz, double *K, double *za_, float *fp, float *fPx, float *fPy, float *fPz,
                             float *fK, float *fza, float *fPA, float *fPB, long long nrec)
{
    const int ip = blockIdx.x * blockDim.x + threadIdx.x;
    if (ip >= npairs) return;
    const int a = psa[ip], b = psb[ip];
    const int Ka = sh_nprim[a], Kb = sh_nprim[b];
    const long long bo = bpoff[key[ip]];
    const bool fwd = a >= b;
    const double *A = xyz + 3 * sh_atom[a], *B = xyz + 3 * sh_atom[b];
    const double AB2 = (A[0] - B[0]) * (A[0] - B[0]) + (A[1] - B[1]) * (A[1] - B[1]) + (A[2] - B[2]) * (A[2] - B[2]);
    int o = poff[ip];
    for (int ka = 0; ka < Ka; ++ka)
        for (int kb = 0; kb < Kb; ++kb) {
            if (!prim_keep(bp, bo, ka, kb, Ka, Kb, fwd, scale, qq, mmax, eps_p)) continue;
            const double za = exps[sh_poff[a] + ka], zb = exps[sh_poff[b] + kb];
            const double p = za + zb;
            const double k = cn[sh_poff[a] + ka] * cn[sh_poff[b] + kb] * exp(-za * zb / p * AB2);
            const double px = (za * A[0] + zb * B[0]) / p, py = (za * A[1] + zb * B[1]) / p,
                         pz = (za * A[2] + zb * B[2]) / p;
            p_[o] = p;
            Px[o] = px;
            Py[o] = py;
            Pz[o] = pz;
            K[o] = k;
            za_[o] = za;
            fp[o] = (float)p;
            fPx[o] = (float)px;
            fPy[o] = (float)py;
            fPz[o] = (float)pz;
            fK[o] = (float)k;
            fza[o] = (float)za;
            fPA[o] = (float)(px - A[0]);
            fPA[nrec + o] = (float)(py - A[1]);
            fPA[2 * nrec + o] = (float)(pz - A[2]);
            fPB[o] = (float)(px - B[0]);
            fPB[nrec + o] = (float)(py - B[1]);
            fPB[2 * nrec + o] = (float)(pz - B[2]);
            ++o;
        }
}

__global__ void k_symm(int nbf, const double *A, double *S)
{
    const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= (long long)nbf * nbf) return;
    const int r = (int)(id / nbf), c = (int)(id % nbf);
    S[id] = A[id] + A[(size_t)c * nbf + r];
}

// Combined density matrices of the Fock build: S_J = sum_p c_J (B_p + B_p^T),
// B_K = sum_p c_K B_p, B_lr = sum_p c_K_lr B_p (pairs in order).
__global__ void k_fock_combine(int nbf, DensArgs den, double *SJ, double *BK, double *BL)
{
    const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= (long long)nbf * nbf) return;
    const int r = (int)(id / nbf), c = (int)(id % nbf);
    double sj = 0.0, bk = 0.0, bl = 0.0;
    for (int p = 0; p < den.npair; ++p) {
        const double v = den.A[p][id], vt = den.A[p][(size_t)c * nbf + r];
        sj += den.cJ[p] * (v + vt);
        bk += den.cK[p] * v;
        bl += den.cKlr[p] * v;
    }
    SJ[id] = sj;
    BK[id] = bk;
    BL[id] = bl;
}

// grad[k] = sum_c partials[c][k] in the fixed order c = 0..nslab-1
__global__ void k_reduce(int n, int nslab, const double *partials, double *grad)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    double s = 0.0;
    for (int c = 0; c < nslab; ++c) s += partials[(size_t)c * n + k];
    grad[k] = s;
}

// Spherical shells (Sec. II.C: the 2l+1 spherical functions of a shell are a
// fixed combination of its Cartesian ones).  With the Cartesian components
// normalised as x^l (every component of a shell carries the same N_k N_c),
// the real solid harmonics of a d shell, each of unit norm, are
//   m = -2: sqrt3 xy   m = -1: sqrt3 yz   m = 0: zz - (xx + yy)/2
//   m = +1: sqrt3 xz   m = +2: (sqrt3/2) (xx - yy),
// so phi_m = sum_c T[c][m] chi_c with the table below (Cartesian order xx,
// xy, xz, yy, yz, zz); s and p shells keep their functions (p: x, y, z).
// A density over spherical functions enters the Cartesian integrals as
// A_cart = T A_sph T^T (T block diagonal over shells), since
// sum (mn|ls)_sph A_mn B_ls = sum (mn|ls)_cart (T A T^T)_mn (T B T^T)_ls.
__device__ const double kSphD[6][5] = {
    {0.0, 0.0, -0.5, 0.0, 0.86602540378443865},   // xx
    {1.7320508075688772, 0.0, 0.0, 0.0, 0.0},      // xy
    {0.0, 0.0, 0.0, 1.7320508075688772, 0.0},      // xz
    {0.0, 0.0, -0.5, 0.0, -0.86602540378443865},  // yy
    {0.0, 1.7320508075688772, 0.0, 0.0, 0.0},      // yz
    {0.0, 0.0, 1.0, 0.0, 0.0}};                    // zz

__device__ __forceinline__ double sph_coef(int l, int c, int m)
{
    return l == 2 ? kSphD[c][m] : (c == m ? 1.0 : 0.0);
}

// One element of A_cart per thread.  cmap[i] for Cartesian function i packs
// the first spherical function of its shell (bits 8..), l (bits 4..7) and its
// Cartesian component (bits 0..3).
__global__ void k_sph_to_cart(int nbf, int nsph, const int *__restrict__ cmap, const double *__restrict__ Asph,
                              double *Acart)
{
    const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= (long long)nbf * nbf) return;
    const int i = (int)(id / nbf), j = (int)(id % nbf);
    const int ci = cmap[i], cj = cmap[j];
    const int si = ci >> 8, li = (ci >> 4) & 15, ki = ci & 15;
    const int sj = cj >> 8, lj = (cj >> 4) & 15, kj = cj & 15;
    const int ni = 2 * li + 1, nj = 2 * lj + 1;
    double acc = 0.0;
    for (int m = 0; m < ni; ++m) {
        const double ti = sph_coef(li, ki, m);
        if (ti == 0.0) continue;
        const double *row = Asph + (size_t)(si + m) * nsph + sj;
        double r = 0.0;
        for (int n = 0; n < nj; ++n) r += row[n] * sph_coef(lj, kj, n);
        acc += ti * r;
    }
    Acart[id] = acc;
}

}  // namespace tg
