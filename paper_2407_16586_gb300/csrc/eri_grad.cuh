// Derivative-ERI class kernels fused with the J/K/K_lr density contraction
// and the per-atom reduction.  One template instance per angular class
// (la lb|lc ld) with la >= lb, lc >= ld and bra pair class >= ket pair class:
// the 21 non-redundant classes for l <= 2 (Sec. II.C).
//
// Per contracted shell quartet (one thread), per primitive quartet, with the
// McMurchie-Davidson expansion
//   (ab|cd) = sum_{h1,h2} E^{ab}_{h1} E^{cd}_{h2} (-1)^{|h2|} R_{h1+h2},
// the derivative of eq. deri is taken as
//   d/dA  : E^{ab} -> DA = 2 zeta_a E^{a+1,b} - a_x E^{a-1,b} (eq. deriv)
//   d/dC  : E^{cd} -> DC likewise
//   d/dA + d/dB = d/dP : R_{h} -> R_{h+1_x}
// and d/dB, d/dD follow from translational invariance (eq. ti).  The density
// contraction (eq. eriupdate summed over a canonical quartet's 8 images) is
// folded in at the half-transformed level:
//   y^{ab}_{h1} = sum_s sum_{h2} [sum_{cd} Gamma_s^{ab,cd} E^{cd}_{h2}] (-1)^{|h2|} R^s_{h1+h2}
//   z^{cd}_{h2} = sum_s sum_{h1} [sum_{ab} Gamma_s^{ab,cd} E^{ab}_{h1}] R^s_{h1+h2}
// with s over the 1/r and erf(w r)/r operators (Gamma_full, Gamma_lr), so
// each gradient component is a short dot product with y or z.
#pragma once
#include "tg_internal.cuh"

namespace tg {

// loop over the Cartesian component pairs of two shells, unrolled (exponents
// are compile-time constants) or not
template <int LX, int LY, bool UNR, typename Fn>
__device__ __forceinline__ void for_pairs(Fn &&fn)
{
    if constexpr (UNR) {
#pragma unroll
        for (int ax = LX; ax >= 0; --ax)
#pragma unroll
            for (int ay = LX - ax; ay >= 0; --ay)
#pragma unroll
                for (int bx = LY; bx >= 0; --bx)
#pragma unroll
                    for (int by = LY - bx; by >= 0; --by)
                        fn(ax, ay, LX - ax - ay, bx, by, LY - bx - by);
    } else {
#pragma unroll 1
        for (int ax = LX; ax >= 0; --ax)
#pragma unroll 1
            for (int ay = LX - ax; ay >= 0; --ay)
#pragma unroll 1
                for (int bx = LY; bx >= 0; --bx)
#pragma unroll 1
                    for (int by = LY - bx; by >= 0; --by)
                        fn(ax, ay, LX - ax - ay, bx, by, LY - bx - by);
    }
}

// Gamma_full and Gamma_lr of the canonical quartet (a b|c d): the sum over
// the 8 permutation images of the ordered density products, times `scale`
// (1/|stabiliser|), summed over the pairs.
template <int LA, int LB, int LC, int LD>
__device__ __forceinline__ void build_gamma(const DensArgs &den, int fa, int fb, int fc, int fd, double scale,
                                            double *gam, double *gaml)
{
    constexpr int NA = ncart(LA), NB = ncart(LB), NC = ncart(LC), ND = ncart(LD);
    constexpr int NCD = NC * ND;
    const int nbf = den.nbf;
    for (int k = 0; k < NA * NB * NCD; ++k) {
        gam[k] = 0.0;
        gaml[k] = 0.0;
    }
    for (int p = 0; p < den.npair; ++p) {
        const double *__restrict__ A = den.A[p];
        const double *__restrict__ B = den.B[p];
        const double *__restrict__ S = den.S[p];
        const double *__restrict__ T = den.T[p];
        const double cj = den.cJ[p] * scale, ck = den.cK[p] * scale, cl = den.cKlr[p] * scale;
        const bool doj = cj != 0.0, dok = (ck != 0.0) || (cl != 0.0);
        if (!doj && !dok) continue;
#pragma unroll 1
        for (int ma = 0; ma < NA; ++ma)
#pragma unroll 1
            for (int mb = 0; mb < NB; ++mb) {
                const size_t m = fa + ma, n = fb + mb;
                const double smn = S[m * nbf + n], tmn = T[m * nbf + n];
#pragma unroll 1
                for (int mc = 0; mc < NC; ++mc)
                    for (int md = 0; md < ND; ++md) {
                        const size_t l = fc + mc, s = fd + md;
                        const int k = (ma * NB + mb) * NCD + mc * ND + md;
                        if (doj) gam[k] += cj * (smn * T[l * nbf + s] + S[l * nbf + s] * tmn);
                        if (dok) {
                            double kk = A[m * nbf + l] * B[n * nbf + s] + A[n * nbf + l] * B[m * nbf + s] +
                                        A[m * nbf + s] * B[n * nbf + l] + A[n * nbf + s] * B[m * nbf + l] +
                                        A[l * nbf + m] * B[s * nbf + n] + A[s * nbf + m] * B[l * nbf + n] +
                                        A[l * nbf + n] * B[s * nbf + m] + A[s * nbf + n] * B[l * nbf + m];
                            gam[k] += ck * kk;
                            gaml[k] += cl * kk;
                        }
                    }
            }
    }
}

// One canonical shell quartet in fp64.  g[12] receives d/dA, d/dB, d/dC, d/dD
// (x, y, z each) of sum Gamma (ab|cd) over both operators.
template <int LA, int LB, int LC, int LD>
__device__ void quartet_fp64(const GeoArgs &geo, const DensArgs &den, const PrimPairs &pp, int sa, int sb, int sc,
                             int sd, int pb0, int nbp, int ib0, int ibs, int pk0, int nkp, double scale,
                             const double *boys, double (&g)[12])
{
    constexpr int NA = ncart(LA), NB = ncart(LB), NC = ncart(LC), ND = ncart(LD);
    constexpr int NAB = NA * NB, NCD = NC * ND;
    constexpr int L1 = LA + LB, L2 = LC + LD, L = L1 + L2;
    constexpr int NH1 = nherm(L1), NH1P = nherm(L1 + 1), NH2 = nherm(L2), NH2P = nherm(L2 + 1);
    constexpr int NR = nherm(L + 1);
    constexpr bool UAB = NAB * NH1P * NH2 <= 64;
    constexpr bool UCD = NCD * NH2P * NH1 <= 64;

    double gam[NAB * NCD], gaml[NAB * NCD];
    build_gamma<LA, LB, LC, LD>(den, geo.sh_bf[sa], geo.sh_bf[sb], geo.sh_bf[sc], geo.sh_bf[sd], scale, gam, gaml);
    const bool lr = den.use_lr;
    const double om2 = den.omega * den.omega;
    const bool ominf = isinf(den.omega);

    const double *xa = geo.xyz + 3 * geo.sh_atom[sa], *xb = geo.xyz + 3 * geo.sh_atom[sb];
    const double *xc = geo.xyz + 3 * geo.sh_atom[sc], *xd = geo.xyz + 3 * geo.sh_atom[sd];
    const double Ax = xa[0], Ay = xa[1], Az = xa[2], Bx = xb[0], By = xb[1], Bz = xb[2];
    const double Cx = xc[0], Cy = xc[1], Cz = xc[2], Dx = xd[0], Dy = xd[1], Dz = xd[2];

    double gA[3] = {0, 0, 0}, gC[3] = {0, 0, 0}, gT[3] = {0, 0, 0};

    for (int ib = ib0; ib < nbp; ib += ibs) {
        const int ip = pb0 + ib;
        const double p = pp.p[ip], Px = pp.Px[ip], Py = pp.Py[ip], Pz = pp.Pz[ip], Kab = pp.K[ip];
        const double za2 = 2.0 * pp.za[ip];
        const double oo2p = 0.5 / p;
        double Ebx[LA + 2][LB + 1][L1 + 2], Eby[LA + 2][LB + 1][L1 + 2], Ebz[LA + 2][LB + 1][L1 + 2];
        etab<LA + 1, LB>(Ebx, Px - Ax, Px - Bx, oo2p);
        etab<LA + 1, LB>(Eby, Py - Ay, Py - By, oo2p);
        etab<LA + 1, LB>(Ebz, Pz - Az, Pz - Bz, oo2p);

        // F_s[cd][h1] = sum_ab Gamma_s[ab][cd] E^{ab}_{h1}
        double Fa[NCD][NH1], Fl[NCD][NH1];
#pragma unroll
        for (int k = 0; k < NCD; ++k)
#pragma unroll
            for (int h = 0; h < NH1; ++h) {
                Fa[k][h] = 0.0;
                Fl[k][h] = 0.0;
            }
        {
            int ab = 0;
            for_pairs<LA, LB, UAB>([&](int ax, int ay, int az, int bx, int by, int bz) {
                for (int t = 0; t <= ax + bx; ++t)
                    for (int u = 0; u <= ay + by; ++u)
                        for (int v = 0; v <= az + bz; ++v) {
                            const double e = Ebx[ax][bx][t] * Eby[ay][by][u] * Ebz[az][bz][v];
                            const int h = hidx(t, u, v);
#pragma unroll
                            for (int k = 0; k < NCD; ++k) {
                                Fa[k][h] += gam[ab * NCD + k] * e;
                                if (lr) Fl[k][h] += gaml[ab * NCD + k] * e;
                            }
                        }
                ++ab;
            });
        }

        for (int jk = 0; jk < nkp; ++jk) {
            const int kp = pk0 + jk;
            const double q = pp.p[kp], Qx = pp.Px[kp], Qy = pp.Py[kp], Qz = pp.Pz[kp], Kcd = pp.K[kp];
            const double zc2 = 2.0 * pp.za[kp];
            const double oo2q = 0.5 / q;
            double Ekx[LC + 2][LD + 1][L2 + 2], Eky[LC + 2][LD + 1][L2 + 2], Ekz[LC + 2][LD + 1][L2 + 2];
            etab<LC + 1, LD>(Ekx, Qx - Cx, Qx - Dx, oo2q);
            etab<LC + 1, LD>(Eky, Qy - Cy, Qy - Dy, oo2q);
            etab<LC + 1, LD>(Ekz, Qz - Cz, Qz - Dz, oo2q);

            // R tensors of both operators, prefactor and contraction coefficients included
            const double pq = p + q;
            const double rho = p * q / pq;
            const double X = Px - Qx, Y = Py - Qy, Z = Pz - Qz;
            const double T = rho * (X * X + Y * Y + Z * Z);
            const double pref = 34.986836655249725 / (p * q * sqrt(pq)) * Kab * Kcd;  // 2 pi^(5/2)
            double R[NR], Rl[NR];
            {
                double Fm[L + 2], base[L + 2];
                boys_fp64<L + 1>(T, Fm, boys);
                double f = pref, m2r = -2.0 * rho;
#pragma unroll
                for (int n = 0; n <= L + 1; ++n) {
                    base[n] = f * Fm[n];
                    f *= m2r;
                }
                hermite_R<L + 1>(R, base, X, Y, Z);
                if (lr) {
                    const double th2 = ominf ? 1.0 : om2 / (om2 + rho);
                    boys_fp64<L + 1>(T * th2, Fm, boys);
                    double fl = pref * sqrt(th2), m2rl = -2.0 * rho * th2;
#pragma unroll
                    for (int n = 0; n <= L + 1; ++n) {
                        base[n] = fl * Fm[n];
                        fl *= m2rl;
                    }
                    hermite_R<L + 1>(Rl, base, X, Y, Z);
                }
            }

            // ket Hermite products E^{cd}_{h2}
            double E3k[NCD][NH2];
            {
                int cd = 0;
                for_pairs<LC, LD, true>([&](int cx, int cy, int cz, int dx, int dy, int dz) {
#pragma unroll
                    for (int h = 0; h < NH2; ++h) E3k[cd][h] = 0.0;
#pragma unroll
                    for (int t = 0; t <= cx + dx; ++t)
#pragma unroll
                        for (int u = 0; u <= cy + dy; ++u)
#pragma unroll
                            for (int v = 0; v <= cz + dz; ++v)
                                E3k[cd][hidx(t, u, v)] = Ekx[cx][dx][t] * Eky[cy][dy][u] * Ekz[cz][dz][v];
                    ++cd;
                });
            }

            // ---- bra side: y^{ab}, then d/dA and d/dP
            {
                int ab = 0;
                for_pairs<LA, LB, UAB>([&](int ax, int ay, int az, int bx, int by, int bz) {
                    double gr[NH2], grl[NH2];
#pragma unroll 1
                    for (int h = 0; h < NH2; ++h) {
                        double s0 = 0.0, s1 = 0.0;
#pragma unroll
                        for (int k = 0; k < NCD; ++k) {
                            s0 += gam[ab * NCD + k] * E3k[k][h];
                            if (lr) s1 += gaml[ab * NCD + k] * E3k[k][h];
                        }
                        gr[h] = s0;
                        grl[h] = s1;
                    }
                    double y[NH1P];
#pragma unroll
                    for (int h = 0; h < NH1P; ++h) y[h] = 0.0;
#pragma unroll 1
                    for (int t2 = 0; t2 <= L2; ++t2)
#pragma unroll 1
                        for (int u2 = 0; u2 <= L2 - t2; ++u2)
#pragma unroll 1
                            for (int v2 = 0; v2 <= L2 - t2 - u2; ++v2) {
                                const int h2 = hidx(t2, u2, v2);
                                const double sg = ((t2 + u2 + v2) & 1) ? -1.0 : 1.0;
                                const double c0 = sg * gr[h2], c1 = sg * grl[h2];
#pragma unroll
                                for (int t1 = 0; t1 <= L1 + 1; ++t1)
#pragma unroll
                                    for (int u1 = 0; u1 <= L1 + 1 - t1; ++u1)
#pragma unroll
                                        for (int v1 = 0; v1 <= L1 + 1 - t1 - u1; ++v1) {
                                            const int hr = hidx(t1 + t2, u1 + u2, v1 + v2);
                                            double acc = y[hidx(t1, u1, v1)] + c0 * R[hr];
                                            if (lr) acc += c1 * Rl[hr];
                                            y[hidx(t1, u1, v1)] = acc;
                                        }
                            }
                    // d/dA and d/dP, factorised over t, u, v with exact ranges
                    const int nx = ax + bx, ny = ay + by, nz = az + bz;
                    double sz[L1 + 2][L1 + 2];  // sz[t][u] = sum_v E_z(v) y[t,u,v]
                    for (int t = 0; t <= nx + 1; ++t)
                        for (int u = 0; u <= ny + 1 && t + u <= L1 + 1; ++u) {
                            double acc = 0.0;
                            for (int v = 0; v <= nz && t + u + v <= L1 + 1; ++v) acc += Ebz[az][bz][v] * y[hidx(t, u, v)];
                            sz[t][u] = acc;
                        }
                    double ax_ = 0.0, ay_ = 0.0, az_ = 0.0, tx = 0.0, ty = 0.0, tz = 0.0;
                    for (int t = 0; t <= nx + 1; ++t) {
                        const double dxt = za2 * Ebx[ax + 1][bx][t] - (ax > 0 ? ax * Ebx[ax - 1][bx][t] : 0.0);
                        double s = 0.0;
                        for (int u = 0; u <= ny; ++u) s += Eby[ay][by][u] * sz[t][u];
                        ax_ += dxt * s;
                    }
                    for (int t = 0; t <= nx; ++t) {
                        const double ext = Ebx[ax][bx][t];
                        double sy = 0.0, sx1 = 0.0, sy1 = 0.0, szd = 0.0, sz1 = 0.0;
                        for (int u = 0; u <= ny + 1; ++u) {
                            const double dyu = za2 * Eby[ay + 1][by][u] - (ay > 0 ? ay * Eby[ay - 1][by][u] : 0.0);
                            sy += dyu * sz[t][u];
                        }
                        for (int u = 0; u <= ny; ++u) {
                            const double eyu = Eby[ay][by][u];
                            sx1 += eyu * sz[t + 1][u];
                            sy1 += eyu * sz[t][u + 1];
                            double a1 = 0.0, a2 = 0.0;
                            for (int v = 0; v <= nz + 1; ++v) {
                                const double dzv = za2 * Ebz[az + 1][bz][v] - (az > 0 ? az * Ebz[az - 1][bz][v] : 0.0);
                                a1 += dzv * y[hidx(t, u, v)];
                            }
                            for (int v = 0; v <= nz; ++v) a2 += Ebz[az][bz][v] * y[hidx(t, u, v + 1)];
                            szd += eyu * a1;
                            sz1 += eyu * a2;
                        }
                        ay_ += ext * sy;
                        az_ += ext * szd;
                        tx += ext * sx1;
                        ty += ext * sy1;
                        tz += ext * sz1;
                    }
                    gA[0] += ax_;
                    gA[1] += ay_;
                    gA[2] += az_;
                    gT[0] += tx;
                    gT[1] += ty;
                    gT[2] += tz;
                    ++ab;
                });
            }

            // ---- ket side: z^{cd}, then d/dC
            {
                int cd = 0;
                for_pairs<LC, LD, UCD>([&](int cx, int cy, int cz, int dx, int dy, int dz) {
                    double z[NH2P];
#pragma unroll
                    for (int h = 0; h < NH2P; ++h) z[h] = 0.0;
#pragma unroll 1
                    for (int t1 = 0; t1 <= L1; ++t1)
#pragma unroll 1
                        for (int u1 = 0; u1 <= L1 - t1; ++u1)
#pragma unroll 1
                            for (int v1 = 0; v1 <= L1 - t1 - u1; ++v1) {
                                const int h1 = hidx(t1, u1, v1);
                                const double f0 = Fa[cd][h1], f1 = Fl[cd][h1];
#pragma unroll
                                for (int t2 = 0; t2 <= L2 + 1; ++t2)
#pragma unroll
                                    for (int u2 = 0; u2 <= L2 + 1 - t2; ++u2)
#pragma unroll
                                        for (int v2 = 0; v2 <= L2 + 1 - t2 - u2; ++v2) {
                                            const int hr = hidx(t1 + t2, u1 + u2, v1 + v2);
                                            double acc = z[hidx(t2, u2, v2)] + f0 * R[hr];
                                            if (lr) acc += f1 * Rl[hr];
                                            z[hidx(t2, u2, v2)] = acc;
                                        }
                            }
                    // d/dC, factorised; the ket sign (-1)^{t+u+v} is folded into z
                    const int nx = cx + dx, ny = cy + dy, nz = cz + dz;
#pragma unroll
                    for (int t2 = 0; t2 <= L2 + 1; ++t2)
#pragma unroll
                        for (int u2 = 0; u2 <= L2 + 1 - t2; ++u2)
#pragma unroll
                            for (int v2 = 0; v2 <= L2 + 1 - t2 - u2; ++v2)
                                if ((t2 + u2 + v2) & 1) z[hidx(t2, u2, v2)] = -z[hidx(t2, u2, v2)];
                    double sz[L2 + 2][L2 + 2];
                    for (int t = 0; t <= nx + 1; ++t)
                        for (int u = 0; u <= ny + 1 && t + u <= L2 + 1; ++u) {
                            double acc = 0.0;
                            for (int v = 0; v <= nz && t + u + v <= L2 + 1; ++v) acc += Ekz[cz][dz][v] * z[hidx(t, u, v)];
                            sz[t][u] = acc;
                        }
                    double cx_ = 0.0, cy_ = 0.0, cz_ = 0.0;
                    for (int t = 0; t <= nx + 1; ++t) {
                        const double dxt = zc2 * Ekx[cx + 1][dx][t] - (cx > 0 ? cx * Ekx[cx - 1][dx][t] : 0.0);
                        double s = 0.0;
                        for (int u = 0; u <= ny; ++u) s += Eky[cy][dy][u] * sz[t][u];
                        cx_ += dxt * s;
                    }
                    for (int t = 0; t <= nx; ++t) {
                        const double ext = Ekx[cx][dx][t];
                        double sy = 0.0, szd = 0.0;
                        for (int u = 0; u <= ny + 1; ++u) {
                            const double dyu = zc2 * Eky[cy + 1][dy][u] - (cy > 0 ? cy * Eky[cy - 1][dy][u] : 0.0);
                            sy += dyu * sz[t][u];
                        }
                        for (int u = 0; u <= ny; ++u) {
                            double a1 = 0.0;
                            for (int v = 0; v <= nz + 1; ++v) {
                                const double dzv = zc2 * Ekz[cz + 1][dz][v] - (cz > 0 ? cz * Ekz[cz - 1][dz][v] : 0.0);
                                a1 += dzv * z[hidx(t, u, v)];
                            }
                            szd += Eky[cy][dy][u] * a1;
                        }
                        cy_ += ext * sy;
                        cz_ += ext * szd;
                    }
                    gC[0] += cx_;
                    gC[1] += cy_;
                    gC[2] += cz_;
                    ++cd;
                });
            }
        }
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        g[i] = gA[i];
        g[3 + i] = gT[i] - gA[i];
        g[6 + i] = gC[i];
        g[9 + i] = -gT[i] - gC[i];
    }
}

// Boys function F_m(T), m = 0..M, for the fp32 route.  Below T = 1 the whole
// fp64 routine runs; for 1 <= T < 36 the top order comes from a Taylor step of
// the fp32 table and the downward recursion F_m = (2T F_{m+1} + e^-T)/(2m+1)
// runs in fp64 (with e^-T in fp64); for T >= 36 the upward recursion is
// stable and runs in fp32.  Relative accuracy ~1e-7 (the fp32 seed).
template <int M>
__device__ __forceinline__ void boys_mixed(float T, float (&F)[M + 1], const double *__restrict__ tab)
{
    if (T < 1.0f) {
        double Fd[M + 1];
        boys_fp64<M>((double)T, Fd, tab);
#pragma unroll
        for (int m = 0; m <= M; ++m) F[m] = (float)Fd[m];
        return;
    }
    if (T < (float)BOYS_TMAX) {
        const float *ftab = reinterpret_cast<const float *>(tab + BOYS_TAB);
        const int i = __float2int_rn(T * (float)(1.0 / BOYS_H));
        const float d = (float)i * (float)BOYS_H - T;
        const float *row = ftab + i * (BOYS_M + 1) + M;
        float acc = row[BOYS_TAYLOR];
#pragma unroll
        for (int k = BOYS_TAYLOR - 1; k >= 0; --k) acc = row[k] + acc * d * (1.0f / (k + 1));
        F[M] = acc;
        const double Td = (double)T;
        const double et = exp(-Td);
        const double t2 = 2.0 * Td;
        double f = (double)acc;
#pragma unroll
        for (int m = M - 1; m >= 0; --m) {
            f = (t2 * f + et) * (1.0 / (2 * m + 1));
            F[m] = (float)f;
        }
    } else {
        const float it = 1.0f / T;
        F[0] = 0.88622692545275801365f * sqrtf(it);
        const float et = __expf(-T);
        const float h = 0.5f * it;
#pragma unroll
        for (int m = 0; m < M; ++m) F[m + 1] = ((2 * m + 1) * F[m] - et) * h;
    }
}

// One canonical shell quartet with fp32 primitive arithmetic.  Same algebra
// as quartet_fp64, in the scaled Hermite basis R'_h = R_h / s^{|h|},
// s = sqrt(2 rho): R'^{(n)}_{000} = pref (-1)^n F_n and the recursion runs
// with X s, so every intermediate stays within fp32 range for any exponent;
// the factors s^{|h|} are moved onto the short Hermite vectors (G rows,
// F rows, y, z) and each bra primitive's contribution is added in fp64.
// Register-resident form: the R tensor, the G row, y and z of
// the current component pair stay in registers: the two operators are
// processed one after the other (one R tensor live at a time), the Hermite
// loops are fully unrolled, and only Gamma / F / E3k rows are read from
// per-thread local memory (one load per row element).  The derivative dot
// products use 1-D rows of the current component pair, zero beyond range.
template <int LA, int LB, int LC, int LD>
__device__ void quartet_fp32r(const GeoArgs &geo, const DensArgs &den, const PrimPairs &pp, int sa, int sb, int sc,
                              int sd, int pb0, int nbp, int ib0, int ibs, int pk0, int nkp, double scale,
                              const double *boys, double (&g)[12])
{
    constexpr int NA = ncart(LA), NB = ncart(LB), NC = ncart(LC), ND = ncart(LD);
    constexpr int NAB = NA * NB, NCD = NC * ND;
    constexpr int L1 = LA + LB, L2 = LC + LD, L = L1 + L2;
    constexpr int NH1 = nherm(L1), NH1P = nherm(L1 + 1), NH2 = nherm(L2), NH2P = nherm(L2 + 1);
    constexpr int NR = nherm(L + 1);
    constexpr int E1 = L1 + 2, E2 = L2 + 2;  // 1-D row lengths

    float gamf[2][NAB * NCD];
    {
        double gd[NAB * NCD], gdl[NAB * NCD];
        build_gamma<LA, LB, LC, LD>(den, geo.sh_bf[sa], geo.sh_bf[sb], geo.sh_bf[sc], geo.sh_bf[sd], scale, gd, gdl);
        for (int k = 0; k < NAB * NCD; ++k) {
            gamf[0][k] = (float)gd[k];
            gamf[1][k] = (float)gdl[k];
        }
    }
    const int nops = den.use_lr ? 2 : 1;
    const float om2f = (float)(den.omega * den.omega);
    const bool ominf = isinf(den.omega);
    const double *xa = geo.xyz + 3 * geo.sh_atom[sa], *xc = geo.xyz + 3 * geo.sh_atom[sc];
    const float ACx = (float)(xa[0] - xc[0]), ACy = (float)(xa[1] - xc[1]), ACz = (float)(xa[2] - xc[2]);
    const long long nr = pp.n;
    double gA[3] = {0, 0, 0}, gC[3] = {0, 0, 0}, gT[3] = {0, 0, 0};

    for (int ib = ib0; ib < nbp; ib += ibs) {
        const int ip = pb0 + ib;
        const float pf = pp.fp[ip], Kab = pp.fK[ip];
        const float PAx = pp.fPA[ip], PAy = pp.fPA[nr + ip], PAz = pp.fPA[2 * nr + ip];
        const float za2 = 2.0f * pp.fza[ip];
        // bra 1-D tables and component rows (local memory: indexed by component)
        float Eb[3][LA + 2][LB + 1][L1 + 2];
        etab<LA + 1, LB>(Eb[0], PAx, pp.fPB[ip], 0.5f / pf);
        etab<LA + 1, LB>(Eb[1], PAy, pp.fPB[nr + ip], 0.5f / pf);
        etab<LA + 1, LB>(Eb[2], PAz, pp.fPB[2 * nr + ip], 0.5f / pf);
        // F_op[cd][h1] = sum_ab Gamma_op[ab][cd] E^{ab}_{h1}
        float Fr[2][NCD][NH1];
        for (int o = 0; o < nops; ++o)
            for (int k = 0; k < NCD; ++k)
#pragma unroll
                for (int h = 0; h < NH1; ++h) Fr[o][k][h] = 0.0f;
        for (int ab = 0; ab < NAB; ++ab) {
            const int ma = ab / NB, mb = ab % NB;
            const int aq = (ma == 0) ? 0 : (ma < 3 ? 1 : 2), bq = (mb == 0) ? 0 : (mb < 3 ? 1 : 2);
            const int ay = aq - (ma - aq * (aq + 1) / 2), ax = LA - aq, az = LA - ax - ay;
            const int by = bq - (mb - bq * (bq + 1) / 2), bx = LB - bq, bz = LB - bx - by;
            float ex[E1], ey[E1], ez[E1];
#pragma unroll
            for (int t = 0; t < E1; ++t) {
                ex[t] = t <= ax + bx ? Eb[0][ax][bx][t] : 0.0f;
                ey[t] = t <= ay + by ? Eb[1][ay][by][t] : 0.0f;
                ez[t] = t <= az + bz ? Eb[2][az][bz][t] : 0.0f;
            }
            float e3[NH1];
#pragma unroll
            for (int t = 0; t <= L1; ++t)
#pragma unroll
                for (int u = 0; u <= L1 - t; ++u)
#pragma unroll
                    for (int v = 0; v <= L1 - t - u; ++v) e3[hidx(t, u, v)] = ex[t] * ey[u] * ez[v];
            for (int o = 0; o < nops; ++o)
                for (int k = 0; k < NCD; ++k) {
                    const float gm = gamf[o][ab * NCD + k];
#pragma unroll
                    for (int h = 0; h < NH1; ++h) Fr[o][k][h] += gm * e3[h];
                }
        }

        // every primitive quartet's contribution is added in fp64
        double fA[3] = {0.0, 0.0, 0.0}, fC[3] = {0.0, 0.0, 0.0}, fT[3] = {0.0, 0.0, 0.0};
        for (int jk = 0; jk < nkp; ++jk) {
            const int kp = pk0 + jk;
            const float qf = pp.fp[kp], Kcd = pp.fK[kp];
            const float QCx = pp.fPA[kp], QCy = pp.fPA[nr + kp], QCz = pp.fPA[2 * nr + kp];
            const float zc2 = 2.0f * pp.fza[kp];
            float Ek[3][LC + 2][LD + 1][L2 + 2];
            etab<LC + 1, LD>(Ek[0], QCx, pp.fPB[kp], 0.5f / qf);
            etab<LC + 1, LD>(Ek[1], QCy, pp.fPB[nr + kp], 0.5f / qf);
            etab<LC + 1, LD>(Ek[2], QCz, pp.fPB[2 * nr + kp], 0.5f / qf);
            const float pq = pf + qf, rho = pf * qf / pq;
            const float Xd = PAx - QCx + ACx, Yd = PAy - QCy + ACy, Zd = PAz - QCz + ACz;
            const float T = rho * (Xd * Xd + Yd * Yd + Zd * Zd);
            const float sc_ = sqrtf(2.0f * rho);
            const float pref = 34.986836655249725f * rsqrtf(pq) / (pf * qf) * Kab * Kcd;
            float spow[L + 3];
            spow[0] = 1.0f;
#pragma unroll
            for (int n = 1; n <= L + 2; ++n) spow[n] = spow[n - 1] * sc_;
            // ket products E^{cd}_{h2} s^{|h2|} (-1)^{|h2|}
            float E3k[NCD][NH2];
            for (int cd = 0; cd < NCD; ++cd) {
                const int mc = cd / ND, md = cd % ND;
                const int cq = (mc == 0) ? 0 : (mc < 3 ? 1 : 2), dq = (md == 0) ? 0 : (md < 3 ? 1 : 2);
                const int cy = cq - (mc - cq * (cq + 1) / 2), cx = LC - cq, cz = LC - cx - cy;
                const int dy = dq - (md - dq * (dq + 1) / 2), dx = LD - dq, dz = LD - dx - dy;
                float kx[E2], ky[E2], kz[E2];
#pragma unroll
                for (int t = 0; t < E2; ++t) {
                    kx[t] = t <= cx + dx ? Ek[0][cx][dx][t] : 0.0f;
                    ky[t] = t <= cy + dy ? Ek[1][cy][dy][t] : 0.0f;
                    kz[t] = t <= cz + dz ? Ek[2][cz][dz][t] : 0.0f;
                }
#pragma unroll
                for (int t = 0; t <= L2; ++t)
#pragma unroll
                    for (int u = 0; u <= L2 - t; ++u)
#pragma unroll
                        for (int v = 0; v <= L2 - t - u; ++v) {
                            const float w = ((t + u + v) & 1) ? -spow[t + u + v] : spow[t + u + v];
                            E3k[cd][hidx(t, u, v)] = kx[t] * ky[u] * kz[v] * w;
                        }
            }
            // this primitive quartet's contribution, formed in fp32, added to fp64 below
            float qA[3] = {0.f, 0.f, 0.f}, qC[3] = {0.f, 0.f, 0.f}, qT[3] = {0.f, 0.f, 0.f};
            for (int o = 0; o < nops; ++o) {
                float R[NR];
                {
                    const float th2 = (o == 0) ? 1.0f : (ominf ? 1.0f : om2f / (om2f + rho));
                    float Fm[L + 2], base[L + 2];
                    boys_mixed<L + 1>(T * th2, Fm, boys);
                    float f = pref * sqrtf(th2);
#pragma unroll
                    for (int n = 0; n <= L + 1; ++n) {
                        base[n] = (n & 1) ? -f * Fm[n] : f * Fm[n];
                        f *= th2;
                    }
                    hermite_R<L + 1>(R, base, Xd * sc_, Yd * sc_, Zd * sc_);
                }
                // ---- bra side: y^{ab} (registers), then d/dA and d/dP
                for (int ab = 0; ab < NAB; ++ab) {
                    float gr[NH2];
#pragma unroll
                    for (int h = 0; h < NH2; ++h) gr[h] = 0.0f;
                    for (int k = 0; k < NCD; ++k) {
                        const float gm = gamf[o][ab * NCD + k];
#pragma unroll
                        for (int h = 0; h < NH2; ++h) gr[h] += gm * E3k[k][h];
                    }
                    float y[NH1P];
#pragma unroll
                    for (int h = 0; h < NH1P; ++h) y[h] = 0.0f;
#pragma unroll
                    for (int t2 = 0; t2 <= L2; ++t2)
#pragma unroll
                        for (int u2 = 0; u2 <= L2 - t2; ++u2)
#pragma unroll
                            for (int v2 = 0; v2 <= L2 - t2 - u2; ++v2) {
                                const float c0 = gr[hidx(t2, u2, v2)];
#pragma unroll
                                for (int t1 = 0; t1 <= L1 + 1; ++t1)
#pragma unroll
                                    for (int u1 = 0; u1 <= L1 + 1 - t1; ++u1)
#pragma unroll
                                        for (int v1 = 0; v1 <= L1 + 1 - t1 - u1; ++v1)
                                            y[hidx(t1, u1, v1)] += c0 * R[hidx(t1 + t2, u1 + u2, v1 + v2)];
                            }
                    const int ma = ab / NB, mb = ab % NB;
                    const int aq = (ma == 0) ? 0 : (ma < 3 ? 1 : 2), bq = (mb == 0) ? 0 : (mb < 3 ? 1 : 2);
                    const int ay = aq - (ma - aq * (aq + 1) / 2), ax = LA - aq, az = LA - ax - ay;
                    const int by = bq - (mb - bq * (bq + 1) / 2), bx = LB - bq, bz = LB - bx - by;
                    // rows: plain E (zero beyond i+j) and derivative DA = 2a E^{i+1} - i E^{i-1}
                    float ex[E1], ey[E1], ez[E1], dx[E1], dy[E1], dz[E1];
#pragma unroll
                    for (int t = 0; t < E1; ++t) {
                        ex[t] = t <= ax + bx ? Eb[0][ax][bx][t] : 0.0f;
                        ey[t] = t <= ay + by ? Eb[1][ay][by][t] : 0.0f;
                        ez[t] = t <= az + bz ? Eb[2][az][bz][t] : 0.0f;
                        dx[t] = za2 * Eb[0][ax + 1][bx][t] - (ax > 0 ? ax * Eb[0][ax - 1][bx][t] : 0.0f);
                        dy[t] = za2 * Eb[1][ay + 1][by][t] - (ay > 0 ? ay * Eb[1][ay - 1][by][t] : 0.0f);
                        dz[t] = za2 * Eb[2][az + 1][bz][t] - (az > 0 ? az * Eb[2][az - 1][bz][t] : 0.0f);
                    }
                    // y_{tuv} s^{t+u+v}, contracted: sum_v (e_z, d_z, shifted e_z) then u, then t
                    float a0 = 0.f, a1 = 0.f, a2 = 0.f, q0 = 0.f, q1 = 0.f, q2 = 0.f;
#pragma unroll
                    for (int t = 0; t <= L1 + 1; ++t) {
                        float ux = 0.f, uy = 0.f, uz = 0.f, vy = 0.f, vz = 0.f;
#pragma unroll
                        for (int u = 0; u <= L1 + 1 - t; ++u) {
                            float sE = 0.f, sD = 0.f, sS = 0.f;
#pragma unroll
                            for (int v = 0; v <= L1 + 1 - t - u; ++v) {
                                const float yy = y[hidx(t, u, v)] * spow[t + u + v];
                                if (v < E1) {
                                    sE += ez[v] * yy;
                                    sD += dz[v] * yy;
                                }
                                if (v >= 1) sS += ez[v - 1] * yy;
                            }
                            ux += ey[u] * sE;  // -> d/dA_x (with dx[t]) and d/dP_x (t-1)
                            uy += dy[u] * sE;  // -> d/dA_y
                            uz += ey[u] * sD;  // -> d/dA_z
                            vz += ey[u] * sS;  // -> d/dP_z
                            if (u >= 1) vy += ey[u - 1] * sE;  // -> d/dP_y
                        }
                        a0 += dx[t] * ux;
                        a1 += ex[t] * uy;
                        a2 += ex[t] * uz;
                        if (t >= 1) q0 += ex[t - 1] * ux;
                        q1 += ex[t] * vy;
                        q2 += ex[t] * vz;
                    }
                    qA[0] += a0;
                    qA[1] += a1;
                    qA[2] += a2;
                    qT[0] += q0;
                    qT[1] += q1;
                    qT[2] += q2;
                }
                // ---- ket side: z^{cd} (registers), then d/dC
                for (int cd = 0; cd < NCD; ++cd) {
                    float z[NH2P];
#pragma unroll
                    for (int h = 0; h < NH2P; ++h) z[h] = 0.0f;
#pragma unroll
                    for (int t1 = 0; t1 <= L1; ++t1)
#pragma unroll
                        for (int u1 = 0; u1 <= L1 - t1; ++u1)
#pragma unroll
                            for (int v1 = 0; v1 <= L1 - t1 - u1; ++v1) {
                                const float f0 = Fr[o][cd][hidx(t1, u1, v1)] * spow[t1 + u1 + v1];
#pragma unroll
                                for (int t2 = 0; t2 <= L2 + 1; ++t2)
#pragma unroll
                                    for (int u2 = 0; u2 <= L2 + 1 - t2; ++u2)
#pragma unroll
                                        for (int v2 = 0; v2 <= L2 + 1 - t2 - u2; ++v2)
                                            z[hidx(t2, u2, v2)] += f0 * R[hidx(t1 + t2, u1 + u2, v1 + v2)];
                            }
                    const int mc = cd / ND, md = cd % ND;
                    const int cq = (mc == 0) ? 0 : (mc < 3 ? 1 : 2), dq = (md == 0) ? 0 : (md < 3 ? 1 : 2);
                    const int cy = cq - (mc - cq * (cq + 1) / 2), cx = LC - cq, cz = LC - cx - cy;
                    const int dy_ = dq - (md - dq * (dq + 1) / 2), dx_ = LD - dq, dz_ = LD - dx_ - dy_;
                    float kx[E2], ky[E2], kz[E2], jx[E2], jy[E2], jz[E2];
#pragma unroll
                    for (int t = 0; t < E2; ++t) {
                        kx[t] = t <= cx + dx_ ? Ek[0][cx][dx_][t] : 0.0f;
                        ky[t] = t <= cy + dy_ ? Ek[1][cy][dy_][t] : 0.0f;
                        kz[t] = t <= cz + dz_ ? Ek[2][cz][dz_][t] : 0.0f;
                        jx[t] = zc2 * Ek[0][cx + 1][dx_][t] - (cx > 0 ? cx * Ek[0][cx - 1][dx_][t] : 0.0f);
                        jy[t] = zc2 * Ek[1][cy + 1][dy_][t] - (cy > 0 ? cy * Ek[1][cy - 1][dy_][t] : 0.0f);
                        jz[t] = zc2 * Ek[2][cz + 1][dz_][t] - (cz > 0 ? cz * Ek[2][cz - 1][dz_][t] : 0.0f);
                    }
                    float c0 = 0.f, c1 = 0.f, c2 = 0.f;
#pragma unroll
                    for (int t = 0; t <= L2 + 1; ++t) {
                        float ux = 0.f, uy = 0.f, uz = 0.f;
#pragma unroll
                        for (int u = 0; u <= L2 + 1 - t; ++u) {
                            float sE = 0.f, sD = 0.f;
#pragma unroll
                            for (int v = 0; v <= L2 + 1 - t - u; ++v) {
                                const int n = t + u + v;
                                const float zz = (n & 1) ? -z[hidx(t, u, v)] * spow[n] : z[hidx(t, u, v)] * spow[n];
                                sE += kz[v] * zz;
                                sD += jz[v] * zz;
                            }
                            ux += ky[u] * sE;
                            uy += jy[u] * sE;
                            uz += ky[u] * sD;
                        }
                        c0 += jx[t] * ux;
                        c1 += kx[t] * uy;
                        c2 += kx[t] * uz;
                    }
                    qC[0] += c0;
                    qC[1] += c1;
                    qC[2] += c2;
                }
            }
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                fA[i] += (double)qA[i];
                fC[i] += (double)qC[i];
                fT[i] += (double)qT[i];
            }
        }
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            gA[i] += fA[i];
            gC[i] += fC[i];
            gT[i] += fT[i];
        }
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        g[i] = gA[i];
        g[3 + i] = gT[i] - gA[i];
        g[6 + i] = gC[i];
        g[9 + i] = -gT[i] - gC[i];
    }
}

// Per-quartet screening bound (see tdgrad.h) and shard membership.
__device__ __forceinline__ bool keep_quartet(const ScreenArgs &scr, const PairSet &bra, const PairSet &ket, int bi,
                                             int ki, int sa, int sb, int sc, int sd)
{
    if (scr.nranks > 1) {
        const int key = max(bra.key[bi], ket.key[ki]);
        if (key % scr.nranks != scr.rank) return false;
    }
    if (scr.tau > 0.0) {
        const double S = fmax(bra.Qd[bi] * ket.Q[ki], bra.Q[bi] * ket.Qd[ki]);
        const int ns = scr.nshell;
        const double *M = scr.M;
        double Mq = M[(size_t)sa * ns + sb];
        Mq = fmax(Mq, M[(size_t)sc * ns + sd]);
        Mq = fmax(Mq, M[(size_t)sa * ns + sc]);
        Mq = fmax(Mq, M[(size_t)sa * ns + sd]);
        Mq = fmax(Mq, M[(size_t)sb * ns + sc]);
        Mq = fmax(Mq, M[(size_t)sb * ns + sd]);
        const double bound = scr.scale * S * Mq * Mq;
        if (bound < scr.tau) return false;
    }
    return true;
}

// Persistent class kernel: CTA c takes tiles c, c+G, c+2G, ... of its class
// (all molecules of a batch; tiles are grouped by molecule).  Every tile's
// 12 x TILE gradient contributions are added to the CTA's partial gradient
// of the current molecule in a fixed order; the partial is flushed to the
// CTA's slab when the molecule changes, so results are bitwise reproducible.
template <int LA, int LB, int LC, int LD, bool FP32>
__global__ void __launch_bounds__(TILE) k_grad(const MolDesc *__restrict__ mols, ClassLaunch cl, OutArgs out,
                                               const double *__restrict__ boys)
{
    extern __shared__ double smem[];
    const int nacc3 = out.use_smem ? out.natom_max * 3 : 0;
    double *sg = smem;
    double *stg = smem + nacc3;
    int *sat = reinterpret_cast<int *>(stg + TILE * 12);
    double *red = reinterpret_cast<double *>(sat + TILE * 4);
    int *ratom = reinterpret_cast<int *>(red + 6 * (TB + TK));
    double *slab = out.partials + (size_t)blockIdx.x * out.natom_total * 3;
    int cur = -1, cur_off3 = 0, cur_n3 = 0;
    unsigned long long nq = 0, npq = 0, nbv = 0;
    // unit = (tile, split): split s takes the bra primitive pairs s, s + S, ...
    const int S = cl.nsplit;
    for (long long it = blockIdx.x; it < cl.ntiles * S; it += gridDim.x) {
        const long long tile = it / S;
        const int split = (int)(it % S);
        const uint4 tl = cl.tiles[tile * cl.stride];
        const int mol = (int)tl.x;
        if (mol != cur) {
            if (out.use_smem) {
                if (cur >= 0)
                    for (int k = threadIdx.x; k < cur_n3; k += blockDim.x) slab[cur_off3 + k] += sg[k];
                __syncthreads();
                for (int k = threadIdx.x; k < nacc3; k += blockDim.x) sg[k] = 0.0;
                __syncthreads();
            }
            cur = mol;
            cur_off3 = mols[mol].atom_off * 3;
            cur_n3 = mols[mol].geo.natom * 3;
        }
        const MolDesc &md = mols[mol];
        const PairSet bra = md.sets[cl.P], ket = md.sets[cl.Q];
        const GeoArgs geo = md.geo;
        const PrimPairs pp = md.pp;
        const ScreenArgs scr = md.scr;
        const bool same = cl.P == cl.Q;
        const int bi = tl.y * TB + threadIdx.x / TK;
        const int ki = tl.z * TK + threadIdx.x % TK;
        double g[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) g[k] = 0.0;
        int at[4] = {-1, -1, -1, -1};
        bool ok = bi < bra.n && ki < ket.n && (!same || bi >= ki);
        if (ok) ok = split < bra.np[bi];
        if (ok) {
            const int sa = bra.sa[bi], sb = bra.sb[bi], sc = ket.sa[ki], sd = ket.sb[ki];
            ok = keep_quartet(scr, bra, ket, bi, ki, sa, sb, sc, sd);
            if (ok) {
                double scale = 1.0;
                if (sa == sb) scale *= 0.5;
                if (sc == sd) scale *= 0.5;
                if (same && bi == ki) scale *= 0.5;
                const int nbp = bra.np[bi], nkp = ket.np[ki];
                if constexpr (FP32)
                    quartet_fp32r<LA, LB, LC, LD>(geo, md.den, pp, sa, sb, sc, sd, bra.poff[bi], nbp, split, S,
                                                  ket.poff[ki], nkp, scale, boys, g);
                else
                    quartet_fp64<LA, LB, LC, LD>(geo, md.den, pp, sa, sb, sc, sd, bra.poff[bi], nbp, split, S,
                                                 ket.poff[ki], nkp, scale, boys, g);
                at[0] = geo.sh_atom[sa];
                at[1] = geo.sh_atom[sb];
                at[2] = geo.sh_atom[sc];
                at[3] = geo.sh_atom[sd];
                if (split == 0) nq += 1;
                npq += (unsigned long long)((nbp - split + S - 1) / S) * nkp;
                nbv += (unsigned long long)((nbp - split + S - 1) / S);
            }
        }
        if (out.dump) {  // dump mode runs with one split per tile
            double *d = out.dump + ((size_t)tile * TILE + threadIdx.x) * 12;
#pragma unroll
            for (int k = 0; k < 12; ++k) d[k] = g[k];
            continue;
        }
#pragma unroll
        for (int k = 0; k < 12; ++k) stg[threadIdx.x * 12 + k] = g[k];
#pragma unroll
        for (int k = 0; k < 4; ++k) sat[threadIdx.x * 4 + k] = at[k];
        __syncthreads();
        tile_reduce(stg, sat, red, ratom, out.use_smem ? sg : slab + cur_off3);
        __syncthreads();
    }
    if (out.use_smem && cur >= 0)
        for (int k = threadIdx.x; k < cur_n3; k += blockDim.x) slab[cur_off3 + k] += sg[k];
    // counters
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        nq += __shfl_xor_sync(0xffffffffu, nq, o);
        npq += __shfl_xor_sync(0xffffffffu, npq, o);
        nbv += __shfl_xor_sync(0xffffffffu, nbv, o);
    }
    if ((threadIdx.x & 31) == 0 && (nq || npq)) {  // a split unit may hold primitives only
        atomicAdd(out.counters + 0, nq);
        atomicAdd(out.counters + (FP32 ? 3 : 1), npq);
        atomicAdd(out.counters + (FP32 ? 5 : 4), nbv);
        if (FP32) atomicAdd(out.counters + 2, nq);
    }
}

// Launch of a persistent class kernel over units: the grid is the smaller of
// gcap and the kernel's resident CTAs per SM times the SM count, and each
// tile is cut into nchunk x nsplit units (nchunk only for the cooperative
// kernel, whose CTA holds ngroups quartets at a time) until there are at
// least four units per CTA, so that classes with few tiles still fill the
// GPU.  Dump mode keeps one unit per tile.
template <typename K>
cudaError_t launch_units(K kern, int ngroups, int gcap, size_t sm, cudaStream_t st, const MolDesc *mols,
                         ClassLaunch cl, const OutArgs &out, const double *boys, int block = TILE)
{
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    int dev = 0, nsm = 1, per = 1;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, block, sm)) != cudaSuccess) return e;
    long long gmax = (long long)(per > 0 ? per : 1) * nsm;
    if (gmax > gcap) gmax = gcap;
    cl.nchunk = 1;
    cl.nsplit = 1;
    if (!out.dump) {
        const long long want = 4 * gmax;
        if (ngroups > 0)
            while (cl.ntiles * cl.nchunk < want && cl.nchunk * ngroups < TILE) cl.nchunk *= 2;
        while (cl.ntiles * cl.nchunk * cl.nsplit < want && cl.nsplit < 4) ++cl.nsplit;
        if (cl.split_req > 0) cl.nsplit = cl.split_req;
    }
    const long long units = cl.ntiles * cl.nchunk * cl.nsplit;
    const int grid = (int)(units < gmax ? units : gmax);
    kern<<<grid, block, sm, st>>>(mols, cl, out, boys);
    return cudaGetLastError();
}

template <int LA, int LB, int LC, int LD>
cudaError_t launch_thread_kernel(int fp32, int gcap, size_t smem, cudaStream_t st, const MolDesc *mols,
                                 const ClassLaunch &cl, const OutArgs &out, const double *boys)
{
    if (fp32) return launch_units(k_grad<LA, LB, LC, LD, true>, 0, gcap, smem, st, mols, cl, out, boys);
    return launch_units(k_grad<LA, LB, LC, LD, false>, 0, gcap, smem, st, mols, cl, out, boys);
}

}  // namespace tg
