// Cooperative derivative-ERI class kernel for the large angular classes.
//
// Same integrals and density contraction as quartet_fp64 / quartet_fp32r
// (eri_grad.cuh), reorganised for a group of GS threads that shares one
// contracted quartet, with every array in shared memory.  Per bra primitive
// pair p and ket primitive pair q (both operators s = full, lr):
//
//   W_s[cd][h1] += sum_h2 (-1)^|h2| E^{cd}_{h2}(q) R_s[h1+h2](p,q)    (over q)
//   z[cd][h2]    = (-1)^|h2| sum_s sum_h1 F_s[cd][h1](p) R_s[h1+h2](p,q)
//   d/dC        += sum_{cd,h2} dE^{cd}_{h2}/dC (q) z[cd][h2]
//
// and after the ket loop Y[ab][h1] = sum_s sum_cd Gamma_s[ab][cd] W_s[cd][h1]
// gives d/dA (with dE^{ab}/dA) and d/dA + d/dB (with E^{ab} and the shifted
// index h1 + 1_x, the R-tensor shift of eq. deriv).  The bra-side density
// contraction therefore happens once per bra primitive pair instead of once
// per primitive quartet, and every phase is split over (function pair,
// Hermite index) items so that all GS threads stay busy.  In fp32 the scaled
// Hermite basis R'_h = R_h / s^{|h|}, s = sqrt(2 rho), keeps values in
// range; the factors s^{|h|} go onto E^{cd}, W and z.
#pragma once
#include "eri_grad.cuh"

namespace tg {

__device__ __forceinline__ void group_sync(int id, int nthreads)
{
    if (nthreads == 32) {
        __syncwarp();
    } else {
        asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
    }
}

template <int LA, int LB, int LC, int LD, typename F>
struct CoopLayout {
    static constexpr int NA = ncart(LA), NB = ncart(LB), NC = ncart(LC), ND = ncart(LD);
    static constexpr int NAB = NA * NB, NCD = NC * ND;
    static constexpr int L1 = LA + LB, L2 = LC + LD, L = L1 + L2;
    static constexpr int NH1 = nherm(L1), NH1P = nherm(L1 + 1), NH2 = nherm(L2), NH2P = nherm(L2 + 1);
    static constexpr int NR = nherm(L + 1);
    static constexpr int NEB = (LA + 2) * (LB + 1) * (L1 + 2);
    static constexpr int NEK = (LC + 2) * (LD + 1) * (L2 + 2);
    // element offsets (in F units) of the per-group regions
    static constexpr int o_gam = 0;
    static constexpr int o_gaml = o_gam + NAB * NCD;
    static constexpr int o_F = o_gaml + NAB * NCD;          // [2][NCD][NH1], per bra primitive pair
    static constexpr int o_E3b = o_F + 2 * NCD * NH1;       // [NAB][NH1], per bra primitive pair
    static constexpr int o_W = o_E3b + NAB * NH1;           // [2][NCD][NH1P], summed over ket primitives
    static constexpr int o_E3k = o_W + 2 * NCD * NH1P;      // [NCD][NH2]
    static constexpr int S = L + 2;                         // dense-cube stride of R
    static constexpr int NCUBE = S * S * S;
    static constexpr int o_R = o_E3k + NCD * NH2;           // [2][S^3] dense R cubes (+ 2 * (L+2) bases)
    static constexpr int o_Eb = o_R + 2 * NCUBE + 2 * (L + 2);  // 3 x NEB
    static constexpr int o_Ek = o_Eb + 3 * NEB;             // 3 x NEK
    static constexpr int o_sc = o_Ek + 3 * NEK;             // scalars and powers of s
    static constexpr int NSC = 16 + L + 3;
    static constexpr int TOTAL = o_sc + NSC;
    static constexpr size_t bytes() { return sizeof(F) * (size_t)TOTAL; }
};

__device__ __forceinline__ int ebi(int i, int j, int t, int J1, int T1) { return (i * J1 + j) * T1 + t; }

// Hermite index h -> (t, u, v), the inverse of hidx.
__device__ __forceinline__ void hdecode(int h, int &n, int &t, int &u, int &v)
{
    n = 0;
    while (nherm(n) <= h) ++n;
    const int r = h - nherm(n - 1);
    int s = 0;
    while ((s + 1) * (s + 2) / 2 <= r) ++s;
    v = r - s * (s + 1) / 2;
    u = s - v;
    t = n - s;
}

// Cartesian component c of a shell of angular momentum l -> exponents
// (lexicographic order xx, xy, xz, yy, yz, zz).
__device__ __forceinline__ void cdecode(int c, int l, int &x, int &y, int &z)
{
    int s = 0;
    while ((s + 1) * (s + 2) / 2 <= c) ++s;
    z = c - s * (s + 1) / 2;
    y = s - z;
    x = l - s;
}

// One contracted quartet by a group of GS threads (lane = thread index within
// the group), bra primitive pairs ib0, ib0 + ibs, ...  Adds this lane's
// partial sums of d/dA (acc[0..2]), d/dA + d/dB (acc[3..5]) and d/dC
// (acc[6..8]); the caller reduces them over the group.
template <int LA, int LB, int LC, int LD, typename F, int GS>
__device__ void quartet_coop(F *sm, int lane, int bar, const GeoArgs &geo, const DensArgs &den, const PrimPairs &pp,
                             int sa, int sb, int sc, int sd, int pb0, int nbp, int ib0, int ibs, int pk0, int nkp,
                             double scale, const double *boys, double (&acc)[9])
{
    using Lay = CoopLayout<LA, LB, LC, LD, F>;
    constexpr int NB = Lay::NB, ND = Lay::ND, NAB = Lay::NAB, NCD = Lay::NCD;
    constexpr int L1 = Lay::L1, L2 = Lay::L2, L = Lay::L;
    constexpr int NH1 = Lay::NH1, NH1P = Lay::NH1P, NH2 = Lay::NH2, NH2P = Lay::NH2P;
    constexpr int BJ = LB + 1, BT = L1 + 2, KJ = LD + 1, KT = L2 + 2;
    constexpr int S = Lay::S, NCUBE = Lay::NCUBE;
    constexpr bool FP32 = sizeof(F) == 4;
    F *gam = sm + Lay::o_gam, *gaml = sm + Lay::o_gaml, *Fr = sm + Lay::o_F, *E3b = sm + Lay::o_E3b;
    F *W = sm + Lay::o_W, *E3k = sm + Lay::o_E3k, *Rb = sm + Lay::o_R, *Eb = sm + Lay::o_Eb, *Ek = sm + Lay::o_Ek;
    F *scl = sm + Lay::o_sc;
    const F *spow = scl + 16;
    const bool lr = den.use_lr;
    const double om2 = den.omega * den.omega;
    const bool ominf = isinf(den.omega);
    const int nbf = den.nbf;
    const int fa = geo.sh_bf[sa], fb = geo.sh_bf[sb], fc = geo.sh_bf[sc], fd = geo.sh_bf[sd];
    const double *xa = geo.xyz + 3 * geo.sh_atom[sa], *xb = geo.xyz + 3 * geo.sh_atom[sb];
    const double *xc = geo.xyz + 3 * geo.sh_atom[sc], *xd = geo.xyz + 3 * geo.sh_atom[sd];

    // ---- Gamma (8 images, scale = 1/|stabiliser|)
    for (int it = lane; it < NAB * NCD; it += GS) {
        const int ab = it / NCD, cd = it % NCD;
        const size_t m = fa + ab / NB, n = fb + ab % NB, l = fc + cd / ND, s = fd + cd % ND;
        double g0 = 0.0, g1 = 0.0;
        for (int p = 0; p < den.npair; ++p) {
            const double *A = den.A[p], *B = den.B[p];
            const double cj = den.cJ[p] * scale, ck = den.cK[p] * scale, cl = den.cKlr[p] * scale;
            if (cj != 0.0)
                g0 += cj * (den.S[p][m * nbf + n] * den.T[p][l * nbf + s] + den.S[p][l * nbf + s] * den.T[p][m * nbf + n]);
            if (ck != 0.0 || cl != 0.0) {
                const double kk = A[m * nbf + l] * B[n * nbf + s] + A[n * nbf + l] * B[m * nbf + s] +
                                  A[m * nbf + s] * B[n * nbf + l] + A[n * nbf + s] * B[m * nbf + l] +
                                  A[l * nbf + m] * B[s * nbf + n] + A[s * nbf + m] * B[l * nbf + n] +
                                  A[l * nbf + n] * B[s * nbf + m] + A[s * nbf + n] * B[l * nbf + m];
                g0 += ck * kk;
                g1 += cl * kk;
            }
        }
        gam[it] = (F)g0;
        gaml[it] = (F)g1;
    }
    group_sync(bar, GS);

    for (int ib = ib0; ib < nbp; ib += ibs) {
        const int ip = pb0 + ib;
        const double p = pp.p[ip], Px = pp.Px[ip], Py = pp.Py[ip], Pz = pp.Pz[ip];
        // 1-D bra Hermite tables, one direction per lane
        if (lane < 3) {
            const double P = lane == 0 ? Px : (lane == 1 ? Py : Pz);
            F E[LA + 2][LB + 1][L1 + 2];
            if constexpr (FP32)
                etab<LA + 1, LB>(E, (F)pp.fPA[lane * pp.n + ip], (F)pp.fPB[lane * pp.n + ip], (F)(0.5f / pp.fp[ip]));
            else
                etab<LA + 1, LB>(E, (F)(P - xa[lane]), (F)(P - xb[lane]), (F)(0.5 / p));
            F *dst = Eb + lane * Lay::NEB;
            for (int i = 0; i <= LA + 1; ++i)
                for (int j = 0; j <= LB; ++j)
                    for (int t = 0; t <= L1 + 1; ++t) dst[ebi(i, j, t, BJ, BT)] = E[i][j][t];
        }
        group_sync(bar, GS);
        // E3b[ab][h1] = E_x E_y E_z (zero outside each component's range); W = 0
        for (int it = lane; it < NAB * NH1; it += GS) {
            const int ab = it / NH1, h = it % NH1;
            int n, t, u, v, ax, ay, az, bx, by, bz;
            hdecode(h, n, t, u, v);
            cdecode(ab / NB, LA, ax, ay, az);
            cdecode(ab % NB, LB, bx, by, bz);
            F e = F(0);
            if (t <= ax + bx && u <= ay + by && v <= az + bz)
                e = Eb[ebi(ax, bx, t, BJ, BT)] * Eb[Lay::NEB + ebi(ay, by, u, BJ, BT)] *
                    Eb[2 * Lay::NEB + ebi(az, bz, v, BJ, BT)];
            E3b[it] = e;
        }
        for (int it = lane; it < 2 * NCD * NH1P; it += GS) W[it] = F(0);
        group_sync(bar, GS);
        // F_s[cd][h1] = sum_ab Gamma_s[ab][cd] E3b[ab][h1]
        for (int it = lane; it < NCD * NH1; it += GS) {
            const int cd = it / NH1, h = it % NH1;
            F s0 = F(0), s1 = F(0);
            for (int ab = 0; ab < NAB; ++ab) {
                const F e = E3b[ab * NH1 + h];
                s0 += gam[ab * NCD + cd] * e;
                s1 += gaml[ab * NCD + cd] * e;
            }
            Fr[it] = s0;
            Fr[NCD * NH1 + it] = s1;
        }
        group_sync(bar, GS);

        for (int jk = 0; jk < nkp; ++jk) {
            const int kp = pk0 + jk;
            // ket tables (lanes 0-2), Boys and R bases (lanes 3, 4)
            if (lane < 3) {
                const double Q = lane == 0 ? pp.Px[kp] : (lane == 1 ? pp.Py[kp] : pp.Pz[kp]);
                F E[LC + 2][LD + 1][L2 + 2];
                if constexpr (FP32)
                    etab<LC + 1, LD>(E, (F)pp.fPA[lane * pp.n + kp], (F)pp.fPB[lane * pp.n + kp],
                                     (F)(0.5f / pp.fp[kp]));
                else
                    etab<LC + 1, LD>(E, (F)(Q - xc[lane]), (F)(Q - xd[lane]), (F)(0.5 / pp.p[kp]));
                F *dst = Ek + lane * Lay::NEK;
                for (int i = 0; i <= LC + 1; ++i)
                    for (int j = 0; j <= LD; ++j)
                        for (int t = 0; t <= L2 + 1; ++t) dst[ebi(i, j, t, KJ, KT)] = E[i][j][t];
            } else if (FP32 && (lane == 3 || (lane == 4 && lr))) {
                // fp32 scalars: P - Q = (P - A) - (Q - C) + (A - C)
                const long long nr = pp.n;
                const float pf = pp.fp[ip], qf = pp.fp[kp], pq = pf + qf, rho = pf * qf / pq;
                const float X = pp.fPA[ip] - pp.fPA[kp] + (float)(xa[0] - xc[0]);
                const float Y = pp.fPA[nr + ip] - pp.fPA[nr + kp] + (float)(xa[1] - xc[1]);
                const float Z = pp.fPA[2 * nr + ip] - pp.fPA[2 * nr + kp] + (float)(xa[2] - xc[2]);
                const float T = rho * (X * X + Y * Y + Z * Z);
                const float pref = 34.986836655249725f * rsqrtf(pq) / (pf * qf) * pp.fK[ip] * pp.fK[kp];
                const float om2f = (float)om2;
                const float th2 = (lane == 3) ? 1.0f : (ominf ? 1.0f : om2f / (om2f + rho));
                float Fm[L + 2];
                boys_mixed<L + 1>(T * th2, Fm, boys);
                F *base = Rb + 2 * NCUBE + (lane - 3) * (L + 2);
                float f = pref * sqrtf(th2);
                for (int n = 0; n <= L + 1; ++n) {
                    base[n] = (F)((n & 1) ? -f * Fm[n] : f * Fm[n]);
                    f *= th2;
                }
                if (lane == 3) {
                    const float s = sqrtf(2.0f * rho);
                    scl[0] = (F)(X * s);
                    scl[1] = (F)(Y * s);
                    scl[2] = (F)(Z * s);
                    F pw = F(1);
                    for (int n = 0; n <= L + 2; ++n) {
                        scl[16 + n] = pw;
                        pw *= (F)s;
                    }
                }
            } else if (!FP32 && (lane == 3 || (lane == 4 && lr))) {
                const double q = pp.p[kp], pq = p + q, rho = p * q / pq;
                const double X = Px - pp.Px[kp], Y = Py - pp.Py[kp], Z = Pz - pp.Pz[kp];
                const double T = rho * (X * X + Y * Y + Z * Z);
                const double pref = 34.986836655249725 / (p * q * sqrt(pq)) * pp.K[ip] * pp.K[kp];
                const double th2 = (lane == 3) ? 1.0 : (ominf ? 1.0 : om2 / (om2 + rho));
                double Fm[L + 2];
                boys_fp64<L + 1>(T * th2, Fm, boys);
                F *base = Rb + 2 * NCUBE + (lane - 3) * (L + 2);
                double f = pref * sqrt(th2), m2 = -2.0 * rho * th2;
                for (int n = 0; n <= L + 1; ++n) {
                    base[n] = (F)(f * Fm[n]);
                    f *= m2;
                }
                if (lane == 3) {
                    scl[0] = (F)X;
                    scl[1] = (F)Y;
                    scl[2] = (F)Z;
                    for (int n = 0; n <= L + 2; ++n) scl[16 + n] = F(1);
                }
            }
            group_sync(bar, GS);
            // R tensors in two dense cubes R3[t][u][v] (stride S), level by
            // level and, within a level, total by total from high to low, so
            // each entry reads level n+1 values (as in hermite_R)
            {
                const F X = scl[0], Y = scl[1], Z = scl[2];
                const int nops = lr ? 2 : 1;
                const F *bases = Rb + 2 * NCUBE;
                if (lane < nops) Rb[lane * NCUBE] = bases[lane * (L + 2) + L + 1];
                group_sync(bar, GS);
                for (int n = L; n >= 0; --n) {
                    for (int k = L + 1 - n; k >= 1; --k) {
                        const int cnt = (k + 1) * (k + 2) / 2;  // triples of total k
                        for (int it = lane; it < nops * cnt; it += GS) {
                            const int o = it / cnt, r = it % cnt;
                            int s = 0;
                            while ((s + 1) * (s + 2) / 2 <= r) ++s;
                            const int v = r - s * (s + 1) / 2, u = s - v, t = k - s;
                            F *c = Rb + o * NCUBE;
                            F val;
                            if (t > 0) {
                                val = X * c[((t - 1) * S + u) * S + v];
                                if (t > 1) val += F(t - 1) * c[((t - 2) * S + u) * S + v];
                            } else if (u > 0) {
                                val = Y * c[(t * S + u - 1) * S + v];
                                if (u > 1) val += F(u - 1) * c[(t * S + u - 2) * S + v];
                            } else {
                                val = Z * c[(t * S + u) * S + v - 1];
                                if (v > 1) val += F(v - 1) * c[(t * S + u) * S + v - 2];
                            }
                            c[(t * S + u) * S + v] = val;
                        }
                        group_sync(bar, GS);
                    }
                    if (lane < nops) Rb[lane * NCUBE] = bases[lane * (L + 2) + n];
                    group_sync(bar, GS);
                }
            }
            const F *R3 = Rb, *R3l = Rb + NCUBE;
            // ket products E3k[cd][h2] = (-1)^|h2| E_x E_y E_z (times s^{|h2|} in fp32)
            for (int it = lane; it < NCD * NH2; it += GS) {
                const int cd = it / NH2, h = it % NH2;
                int n, t, u, v, cx, cy, cz, dx, dy, dz;
                hdecode(h, n, t, u, v);
                cdecode(cd / ND, LC, cx, cy, cz);
                cdecode(cd % ND, LD, dx, dy, dz);
                F e = F(0);
                if (t <= cx + dx && u <= cy + dy && v <= cz + dz)
                    e = Ek[ebi(cx, dx, t, KJ, KT)] * Ek[Lay::NEK + ebi(cy, dy, u, KJ, KT)] *
                        Ek[2 * Lay::NEK + ebi(cz, dz, v, KJ, KT)] * spow[n];
                E3k[it] = (n & 1) ? -e : e;
            }
            group_sync(bar, GS);
            // W_s[cd][h1] += s^{|h1|} sum_h2 E3k[cd][h2] R_s[h1+h2]; the cube
            // index of h1+h2 is base(h1) + off(h2), off a constant of the
            // unrolled h2 loop
            for (int it = lane; it < NCD * NH1P; it += GS) {
                const int cd = it / NH1P, h1 = it % NH1P;
                int n1, t1, u1, v1;
                hdecode(h1, n1, t1, u1, v1);
                const int b1 = (t1 * S + u1) * S + v1;
                const F *e = E3k + cd * NH2;
                F w0 = F(0), w1 = F(0);
#pragma unroll
                for (int t2 = 0; t2 <= L2; ++t2)
#pragma unroll
                    for (int u2 = 0; u2 <= L2 - t2; ++u2)
#pragma unroll
                        for (int v2 = 0; v2 <= L2 - t2 - u2; ++v2) {
                            const int off = (t2 * S + u2) * S + v2;
                            const F ev = e[hidx(t2, u2, v2)];
                            w0 += ev * R3[b1 + off];
                            if (lr) w1 += ev * R3l[b1 + off];
                        }
                if constexpr (FP32) {
                    w0 *= spow[n1];
                    w1 *= spow[n1];
                }
                W[it] += w0;
                if (lr) W[NCD * NH1P + it] += w1;
            }
            // z[cd][h2] = (-1)^|h2| s^{|h2|} sum_s sum_h1 F_s[cd][h1] s^{|h1|} R_s[h1+h2],
            // contracted at once with dE^{cd}_{h2}/dC
            {
                const F zc2 = (F)(2.0 * pp.za[kp]);
                const F *Ex = Ek, *Ey = Ek + Lay::NEK, *Ez = Ek + 2 * Lay::NEK;
                F c0 = F(0), c1 = F(0), c2 = F(0);
                for (int it = lane; it < NCD * NH2P; it += GS) {
                    const int cd = it / NH2P, h2 = it % NH2P;
                    int n2, t2, u2, v2, cx, cy, cz, dx, dy, dz;
                    hdecode(h2, n2, t2, u2, v2);
                    cdecode(cd / ND, LC, cx, cy, cz);
                    cdecode(cd % ND, LD, dx, dy, dz);
                    const int nx = cx + dx, ny = cy + dy, nz = cz + dz;
                    if (t2 > nx + 1 || u2 > ny + 1 || v2 > nz + 1) continue;
                    const int b2 = (t2 * S + u2) * S + v2;
                    const F *f0 = Fr + cd * NH1, *f1 = Fr + NCD * NH1 + cd * NH1;
                    F z0 = F(0), z1 = F(0);
#pragma unroll
                    for (int t1 = 0; t1 <= L1; ++t1)
#pragma unroll
                        for (int u1 = 0; u1 <= L1 - t1; ++u1)
#pragma unroll
                            for (int v1 = 0; v1 <= L1 - t1 - u1; ++v1) {
                                const int off = (t1 * S + u1) * S + v1;
                                if constexpr (FP32) {
                                    const F sh = spow[t1 + u1 + v1];
                                    z0 += f0[hidx(t1, u1, v1)] * sh * R3[b2 + off];
                                    if (lr) z1 += f1[hidx(t1, u1, v1)] * sh * R3l[b2 + off];
                                } else {
                                    z0 += f0[hidx(t1, u1, v1)] * R3[b2 + off];
                                    if (lr) z1 += f1[hidx(t1, u1, v1)] * R3l[b2 + off];
                                }
                            }
                    F z = z0 + z1;
                    if constexpr (FP32) z *= spow[n2];
                    if (n2 & 1) z = -z;
                    const F ex = t2 <= nx ? Ex[ebi(cx, dx, t2, KJ, KT)] : F(0);
                    const F ey = u2 <= ny ? Ey[ebi(cy, dy, u2, KJ, KT)] : F(0);
                    const F ez = v2 <= nz ? Ez[ebi(cz, dz, v2, KJ, KT)] : F(0);
                    if (u2 <= ny && v2 <= nz) {
                        const F dxv = zc2 * Ex[ebi(cx + 1, dx, t2, KJ, KT)] -
                                      (cx > 0 ? F(cx) * Ex[ebi(cx - 1, dx, t2, KJ, KT)] : F(0));
                        c0 += dxv * ey * ez * z;
                    }
                    if (t2 <= nx && v2 <= nz) {
                        const F dyv = zc2 * Ey[ebi(cy + 1, dy, u2, KJ, KT)] -
                                      (cy > 0 ? F(cy) * Ey[ebi(cy - 1, dy, u2, KJ, KT)] : F(0));
                        c1 += ex * dyv * ez * z;
                    }
                    if (t2 <= nx && u2 <= ny) {
                        const F dzv = zc2 * Ez[ebi(cz + 1, dz, v2, KJ, KT)] -
                                      (cz > 0 ? F(cz) * Ez[ebi(cz - 1, dz, v2, KJ, KT)] : F(0));
                        c2 += ex * ey * dzv * z;
                    }
                }
                acc[6] += (double)c0;
                acc[7] += (double)c1;
                acc[8] += (double)c2;
            }
            group_sync(bar, GS);
        }

        // Y[ab][h1] = sum_s sum_cd Gamma_s[ab][cd] W_s[cd][h1], contracted at once
        // with dE^{ab}_{h1}/dA (d/dA) and with E^{ab}_{h1 - 1_x} (d/dA + d/dB)
        {
            const F za2 = (F)(2.0 * pp.za[ip]);
            const F *Ex = Eb, *Ey = Eb + Lay::NEB, *Ez = Eb + 2 * Lay::NEB;
            F a0 = F(0), a1 = F(0), a2 = F(0), q0 = F(0), q1 = F(0), q2 = F(0);
            for (int it = lane; it < NAB * NH1P; it += GS) {
                const int ab = it / NH1P, h1 = it % NH1P;
                int n1, t, u, v, ax, ay, az, bx, by, bz;
                hdecode(h1, n1, t, u, v);
                cdecode(ab / NB, LA, ax, ay, az);
                cdecode(ab % NB, LB, bx, by, bz);
                const int nx = ax + bx, ny = ay + by, nz = az + bz;
                if (t > nx + 1 || u > ny + 1 || v > nz + 1) continue;
                const F *g0 = gam + ab * NCD, *g1 = gaml + ab * NCD;
                F y = F(0);
                for (int cd = 0; cd < NCD; ++cd) {
                    y += g0[cd] * W[cd * NH1P + h1];
                    if (lr) y += g1[cd] * W[(NCD + cd) * NH1P + h1];
                }
                const F ex = t <= nx ? Ex[ebi(ax, bx, t, BJ, BT)] : F(0);
                const F ey = u <= ny ? Ey[ebi(ay, by, u, BJ, BT)] : F(0);
                const F ez = v <= nz ? Ez[ebi(az, bz, v, BJ, BT)] : F(0);
                if (u <= ny && v <= nz) {
                    const F dxv = za2 * Ex[ebi(ax + 1, bx, t, BJ, BT)] -
                                  (ax > 0 ? F(ax) * Ex[ebi(ax - 1, bx, t, BJ, BT)] : F(0));
                    a0 += dxv * ey * ez * y;
                    if (t >= 1 && t - 1 <= nx) q0 += Ex[ebi(ax, bx, t - 1, BJ, BT)] * ey * ez * y;
                }
                if (t <= nx && v <= nz) {
                    const F dyv = za2 * Ey[ebi(ay + 1, by, u, BJ, BT)] -
                                  (ay > 0 ? F(ay) * Ey[ebi(ay - 1, by, u, BJ, BT)] : F(0));
                    a1 += ex * dyv * ez * y;
                    if (u >= 1 && u - 1 <= ny) q1 += ex * Ey[ebi(ay, by, u - 1, BJ, BT)] * ez * y;
                }
                if (t <= nx && u <= ny) {
                    const F dzv = za2 * Ez[ebi(az + 1, bz, v, BJ, BT)] -
                                  (az > 0 ? F(az) * Ez[ebi(az - 1, bz, v, BJ, BT)] : F(0));
                    a2 += ex * ey * dzv * y;
                    if (v >= 1 && v - 1 <= nz) q2 += ex * ey * Ez[ebi(az, bz, v - 1, BJ, BT)] * y;
                }
            }
            acc[0] += (double)a0;
            acc[1] += (double)a1;
            acc[2] += (double)a2;
            acc[3] += (double)q0;
            acc[4] += (double)q1;
            acc[5] += (double)q2;
        }
        group_sync(bar, GS);
    }
}

// Persistent cooperative class kernel: 128 threads = 128/GS groups; group g
// takes quartets g, g + 128/GS, ... of every tile; the tile's 12 x TILE
// contributions are then added in the same fixed order as k_grad.
template <int LA, int LB, int LC, int LD, typename F, int GS>
__global__ void __launch_bounds__(TILE) k_grad_coop(const MolDesc *__restrict__ mols, ClassLaunch cl, OutArgs out,
                                                    const double *__restrict__ boys)
{
    using Lay = CoopLayout<LA, LB, LC, LD, F>;
    constexpr int NG = TILE / GS;
    extern __shared__ double smem[];
    const int nacc3 = out.use_smem ? out.natom_max * 3 : 0;
    double *sg = smem;
    double *stg = smem + nacc3;
    int *sat = reinterpret_cast<int *>(stg + TILE * 12);
    double *tred = reinterpret_cast<double *>(sat + TILE * 4);
    int *ratom = reinterpret_cast<int *>(tred + 6 * (TB + TK));
    double *red = reinterpret_cast<double *>(ratom + 2 * (TB + TK));  // [NG][GS/32][9]
    F *gsm = reinterpret_cast<F *>(red + NG * (GS / 32) * 9) + (size_t)(threadIdx.x / GS) * Lay::TOTAL;
    const int grp = threadIdx.x / GS, lane = threadIdx.x % GS, bar = 1 + grp;
    double *slab = out.partials + (size_t)blockIdx.x * out.natom_total * 3;
    int cur = -1, cur_off3 = 0, cur_n3 = 0;
    unsigned long long nq = 0, npq = 0, nbv = 0;
    // unit = (tile, chunk, split): chunk c holds quartets c * QPC ... of the
    // tile, split s takes the bra primitive pairs s, s + S, ...
    const int S = cl.nsplit, C = cl.nchunk, QPC = TILE / C;
    for (long long it = blockIdx.x; it < cl.ntiles * C * S; it += gridDim.x) {
        const long long tile = it / (C * S);
        const int chunk = (int)((it / S) % C), split = (int)(it % S);
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
        if (C > 1 && !out.dump) {
            for (int k = threadIdx.x; k < TILE * 12; k += blockDim.x) stg[k] = 0.0;
            for (int k = threadIdx.x; k < TILE * 4; k += blockDim.x) sat[k] = -1;
            __syncthreads();
        }
        for (int qi = chunk * QPC + grp; qi < (chunk + 1) * QPC; qi += NG) {
            const int bi = tl.y * TB + qi / TK;
            const int ki = tl.z * TK + qi % TK;
            double g[12];
#pragma unroll
            for (int k = 0; k < 12; ++k) g[k] = 0.0;
            int at[4] = {-1, -1, -1, -1};
            bool ok = bi < bra.n && ki < ket.n && (!same || bi >= ki);
            if (ok) ok = split < bra.np[bi];
            int sa = 0, sb = 0, sc = 0, sd = 0;
            if (ok) {
                sa = bra.sa[bi];
                sb = bra.sb[bi];
                sc = ket.sa[ki];
                sd = ket.sb[ki];
                ok = keep_quartet(scr, bra, ket, bi, ki, sa, sb, sc, sd);
            }
            if (ok) {  // uniform across the group
                double scale = 1.0;
                if (sa == sb) scale *= 0.5;
                if (sc == sd) scale *= 0.5;
                if (same && bi == ki) scale *= 0.5;
                const int nbp = bra.np[bi], nkp = ket.np[ki];
                double acc[9];
#pragma unroll
                for (int k = 0; k < 9; ++k) acc[k] = 0.0;
                quartet_coop<LA, LB, LC, LD, F, GS>(gsm, lane, bar, geo, md.den, pp, sa, sb, sc, sd, bra.poff[bi],
                                                    nbp, split, S, ket.poff[ki], nkp, scale, boys, acc);
#pragma unroll
                for (int k = 0; k < 9; ++k)
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], o);
                double *rg = red + (size_t)grp * (GS / 32) * 9;
                if ((lane & 31) == 0)
#pragma unroll
                    for (int k = 0; k < 9; ++k) rg[(lane / 32) * 9 + k] = acc[k];
                group_sync(bar, GS);
                if (lane == 0) {
                    double s9[9];
#pragma unroll
                    for (int k = 0; k < 9; ++k) {
                        double s = 0.0;
                        for (int w = 0; w < GS / 32; ++w) s += rg[w * 9 + k];
                        s9[k] = s;
                    }
#pragma unroll
                    for (int i = 0; i < 3; ++i) {
                        g[i] = s9[i];
                        g[3 + i] = s9[3 + i] - s9[i];
                        g[6 + i] = s9[6 + i];
                        g[9 + i] = -s9[3 + i] - s9[6 + i];
                    }
                    at[0] = geo.sh_atom[sa];
                    at[1] = geo.sh_atom[sb];
                    at[2] = geo.sh_atom[sc];
                    at[3] = geo.sh_atom[sd];
                    if (split == 0) nq += 1;
                    npq += (unsigned long long)((nbp - split + S - 1) / S) * nkp;
                    nbv += (unsigned long long)((nbp - split + S - 1) / S);
                }
                group_sync(bar, GS);
            }
            if (lane == 0) {
                if (out.dump) {
                    double *d = out.dump + ((size_t)tile * TILE + qi) * 12;  // one unit per tile
#pragma unroll
                    for (int k = 0; k < 12; ++k) d[k] = g[k];
                } else {
#pragma unroll
                    for (int k = 0; k < 12; ++k) stg[qi * 12 + k] = g[k];
#pragma unroll
                    for (int k = 0; k < 4; ++k) sat[qi * 4 + k] = at[k];
                }
            }
        }
        __syncthreads();
        if (!out.dump) tile_reduce(stg, sat, tred, ratom, out.use_smem ? sg : slab + cur_off3);
        __syncthreads();
    }
    if (out.use_smem && cur >= 0)
        for (int k = threadIdx.x; k < cur_n3; k += blockDim.x) slab[cur_off3 + k] += sg[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        nq += __shfl_xor_sync(0xffffffffu, nq, o);
        npq += __shfl_xor_sync(0xffffffffu, npq, o);
        nbv += __shfl_xor_sync(0xffffffffu, nbv, o);
    }
    if ((threadIdx.x & 31) == 0 && (nq || npq)) {  // a split unit may hold primitives only
        atomicAdd(out.counters + 0, nq);
        atomicAdd(out.counters + (sizeof(F) == 4 ? 3 : 1), npq);
        atomicAdd(out.counters + (sizeof(F) == 4 ? 5 : 4), nbv);
        if (sizeof(F) == 4) atomicAdd(out.counters + 2, nq);
    }
}

// Group size and shared-memory use of the cooperative kernel for a class.
template <int LA, int LB, int LC, int LD, typename F>
struct CoopChoice {
    using Lay = CoopLayout<LA, LB, LC, LD, F>;
    static constexpr int work = Lay::NAB * Lay::NH1P > Lay::NCD * Lay::NH2P ? Lay::NAB * Lay::NH1P : Lay::NCD * Lay::NH2P;
    static constexpr int GS = work >= 1024 ? 128 : (work >= 320 ? 64 : 32);
    static constexpr size_t group_bytes() { return Lay::bytes(); }
    static constexpr size_t bytes_all() { return (size_t)(TILE / GS) * Lay::bytes() + sizeof(double) * (TILE / GS) * (GS / 32) * 9 + 64; }
};

}  // namespace tg

namespace tg {

template <int LA, int LB, int LC, int LD, typename F>
cudaError_t launch_coop(int gcap, size_t smem, cudaStream_t st, const MolDesc *mols, const ClassLaunch &cl,
                        const OutArgs &out, const double *boys)
{
    using C = CoopChoice<LA, LB, LC, LD, F>;
    return launch_units(k_grad_coop<LA, LB, LC, LD, F, C::GS>, TILE / C::GS, gcap, smem + C::bytes_all(), st, mols,
                        cl, out, boys);
}

}  // namespace tg
