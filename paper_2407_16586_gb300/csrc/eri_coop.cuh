// Cooperative derivative-ERI class kernel for the large angular classes.
//
// Same algebra as quartet_fp64 / quartet_fp32 (eri_grad.cuh), but a group of
// GS threads shares one contracted quartet and every array lives in shared
// memory: Gamma, the F rows (per bra primitive pair), the ket Hermite
// products, the R tensors, the G rows, and y / z.  Each phase is split over
// (function pair, Hermite index) items, so a d-shell quartet keeps all GS
// threads busy without spilling to local memory.  In fp32 the scaled Hermite
// basis R'_h = R_h / s^{|h|}, s = sqrt(2 rho), keeps values in range.
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
    static constexpr int o_F = o_gaml + NAB * NCD;          // [2][NCD][NH1]
    static constexpr int o_E3k = o_F + 2 * NCD * NH1;       // [NCD][NH2]
    static constexpr int S = L + 2;                         // dense-cube stride of R
    static constexpr int NCUBE = S * S * S;
    static constexpr int o_R = o_E3k + NCD * NH2;           // [2][S^3] dense R cubes (+ 2 * (L+2) bases)
    static constexpr int o_G = o_R + 2 * NCUBE + 2 * (L + 2);  // [2][NAB][NH2]; E3b [NAB][NH1] aliases it
    static constexpr int GSZ = 2 * NAB * NH2 > NAB * NH1 ? 2 * NAB * NH2 : NAB * NH1;
    static constexpr int o_YZ = o_G + GSZ;                  // y [NAB][NH1P] or z [NCD][NH2P]
    static constexpr int YZ = NAB * NH1P > NCD * NH2P ? NAB * NH1P : NCD * NH2P;
    static constexpr int o_Eb = o_YZ + YZ;                  // 3 x NEB
    static constexpr int o_Ek = o_Eb + 3 * NEB;             // 3 x NEK
    static constexpr int o_sc = o_Ek + 3 * NEK;             // scalars and powers of s
    static constexpr int NSC = 16 + L + 3;
    static constexpr int TOTAL = o_sc + NSC;
    static constexpr size_t bytes() { return sizeof(F) * (size_t)TOTAL; }
};

__device__ __forceinline__ int ebi(int i, int j, int t, int J1, int T1) { return (i * J1 + j) * T1 + t; }

// One contracted quartet by a group of GS threads (lane = thread index within
// the group).  Returns d/dA, d/dP, d/dC partial sums of this lane; the caller
// reduces them over the group.
template <int LA, int LB, int LC, int LD, typename F, int GS>
__device__ void quartet_coop(F *sm, int lane, int bar, const GeoArgs &geo, const DensArgs &den, const PrimPairs &pp,
                             int sa, int sb, int sc, int sd, int pb0, int nbp, int ib0, int ibs, int pk0, int nkp,
                             double scale, const double *boys, double (&acc)[9])
{
    using Lay = CoopLayout<LA, LB, LC, LD, F>;
    constexpr int NB = Lay::NB, ND = Lay::ND, NAB = Lay::NAB, NCD = Lay::NCD;
    constexpr int L1 = Lay::L1, L2 = Lay::L2, L = Lay::L;
    constexpr int NH1 = Lay::NH1, NH1P = Lay::NH1P, NH2 = Lay::NH2, NH2P = Lay::NH2P, NR = Lay::NR;
    constexpr int BJ = LB + 1, BT = L1 + 2, KJ = LD + 1, KT = L2 + 2;
    constexpr bool FP32 = sizeof(F) == 4;
    F *gam = sm + Lay::o_gam, *gaml = sm + Lay::o_gaml, *Fr = sm + Lay::o_F, *E3k = sm + Lay::o_E3k;
    F *Rb = sm + Lay::o_R, *G = sm + Lay::o_G, *YZ = sm + Lay::o_YZ, *Eb = sm + Lay::o_Eb, *Ek = sm + Lay::o_Ek;
    F *scl = sm + Lay::o_sc;
    F *E3b = G;  // aliases G: only used while building the F rows
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
        // E3b[ab][h1] = E_x E_y E_z (zero outside each component's range)
        for (int it = lane; it < NAB * NH1; it += GS) {
            const int ab = it / NH1, h = it % NH1;
            int t, u, v;
            {
                int n = 0;
                while (nherm(n) <= h) ++n;
                const int r = h - nherm(n - 1);
                int s = 0;
                while ((s + 1) * (s + 2) / 2 <= r) ++s;
                v = r - s * (s + 1) / 2;
                u = s - v;
                t = n - s;
            }
            const int ma = ab / NB, mb = ab % NB;
            int ax, ay, bx, by;
            {
                // component -> exponents (lexicographic order)
                int c = ma, l = LA, s = 0;
                while ((s + 1) * (s + 2) / 2 <= c) ++s;
                const int lz = c - s * (s + 1) / 2;
                ay = s - lz;
                ax = l - s;
                c = mb;
                l = LB;
                s = 0;
                while ((s + 1) * (s + 2) / 2 <= c) ++s;
                const int lz2 = c - s * (s + 1) / 2;
                by = s - lz2;
                bx = l - s;
            }
            const int az = LA - ax - ay, bz = LB - bx - by;
            F e = F(0);
            if (t <= ax + bx && u <= ay + by && v <= az + bz)
                e = Eb[ebi(ax, bx, t, BJ, BT)] * Eb[Lay::NEB + ebi(ay, by, u, BJ, BT)] *
                    Eb[2 * Lay::NEB + ebi(az, bz, v, BJ, BT)];
            E3b[it] = e;
        }
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
                F *base = Rb + 2 * Lay::NCUBE + (lane - 3) * (L + 2);
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
                F *base = Rb + 2 * Lay::NCUBE + (lane - 3) * (L + 2);
                if (FP32) {
                    // scaled basis: base'_n = pref theta (-theta^2)^n F_n, recursion with X s
                    double f = pref * sqrt(th2);
                    for (int n = 0; n <= L + 1; ++n) {
                        base[n] = (F)((n & 1) ? -f * Fm[n] : f * Fm[n]);
                        f *= th2;
                    }
                    if (lane == 3) {
                        const double s = sqrt(2.0 * rho);
                        scl[0] = (F)(X * s);
                        scl[1] = (F)(Y * s);
                        scl[2] = (F)(Z * s);
                        F pw = F(1);
                        for (int n = 0; n <= L + 2; ++n) {
                            scl[16 + n] = pw;
                            pw *= (F)s;
                        }
                    }
                } else {
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
            }
            group_sync(bar, GS);
            // R tensors in two dense cubes R3[t][u][v] (stride S), level by
            // level and, within a level, total by total from high to low, so
            // each entry reads level n+1 values (as in hermite_R)
            {
                constexpr int S = Lay::S, NCUBE = Lay::NCUBE;
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
            constexpr int S = Lay::S;
            const F *R3 = Rb, *R3l = Rb + Lay::NCUBE;
            const F *spow = scl + 16;
            // ket products E3k[cd][h2] (times s^{|h2|} in fp32)
            for (int it = lane; it < NCD * NH2; it += GS) {
                const int cd = it / NH2, h = it % NH2;
                int n = 0;
                while (nherm(n) <= h) ++n;
                const int rr = h - nherm(n - 1);
                int s = 0;
                while ((s + 1) * (s + 2) / 2 <= rr) ++s;
                const int v = rr - s * (s + 1) / 2, u = s - v, t = n - s;
                const int mc = cd / ND, md = cd % ND;
                int cx, cy, dx, dy;
                {
                    int c = mc, q = 0;
                    while ((q + 1) * (q + 2) / 2 <= c) ++q;
                    cy = q - (c - q * (q + 1) / 2);
                    cx = LC - q;
                    c = md;
                    q = 0;
                    while ((q + 1) * (q + 2) / 2 <= c) ++q;
                    dy = q - (c - q * (q + 1) / 2);
                    dx = LD - q;
                }
                const int cz = LC - cx - cy, dz = LD - dx - dy;
                F e = F(0);
                if (t <= cx + dx && u <= cy + dy && v <= cz + dz)
                    e = Ek[ebi(cx, dx, t, KJ, KT)] * Ek[Lay::NEK + ebi(cy, dy, u, KJ, KT)] *
                        Ek[2 * Lay::NEK + ebi(cz, dz, v, KJ, KT)] * spow[n];
                E3k[it] = e;
            }
            group_sync(bar, GS);
            // G_s[ab][h2] = sum_cd Gamma_s[ab][cd] E3k[cd][h2], times (-1)^{|h2|}
            for (int it = lane; it < NAB * NH2; it += GS) {
                const int ab = it / NH2, h = it % NH2;
                F s0 = F(0), s1 = F(0);
                for (int cd = 0; cd < NCD; ++cd) {
                    const F e = E3k[cd * NH2 + h];
                    s0 += gam[ab * NCD + cd] * e;
                    s1 += gaml[ab * NCD + cd] * e;
                }
                int n = 0;
                while (nherm(n) <= h) ++n;
                if (n & 1) {
                    s0 = -s0;
                    s1 = -s1;
                }
                G[it] = s0;
                G[NAB * NH2 + it] = s1;
            }
            group_sync(bar, GS);
            // y[ab][h1] = sum_h2 G[ab][h2] R[h1+h2] (+ lr), times s^{|h1|}; the
            // cube index of h1+h2 is base(h1) + off(h2) with off a constant of
            // the unrolled h2 loop
            for (int it = lane; it < NAB * NH1P; it += GS) {
                const int ab = it / NH1P, h1 = it % NH1P;
                int n1 = 0;
                while (nherm(n1) <= h1) ++n1;
                const int r1 = h1 - nherm(n1 - 1);
                int s1 = 0;
                while ((s1 + 1) * (s1 + 2) / 2 <= r1) ++s1;
                const int v1 = r1 - s1 * (s1 + 1) / 2, u1 = s1 - v1, t1 = n1 - s1;
                const int b1 = (t1 * S + u1) * S + v1;
                const F *g0 = G + ab * NH2, *g1 = G + NAB * NH2 + ab * NH2;
                F y0 = F(0), y1 = F(0);
#pragma unroll
                for (int t2 = 0; t2 <= L2; ++t2)
#pragma unroll
                    for (int u2 = 0; u2 <= L2 - t2; ++u2)
#pragma unroll
                        for (int v2 = 0; v2 <= L2 - t2 - u2; ++v2) {
                            const int off = (t2 * S + u2) * S + v2;
                            y0 += g0[hidx(t2, u2, v2)] * R3[b1 + off];
                            if (lr) y1 += g1[hidx(t2, u2, v2)] * R3l[b1 + off];
                        }
                F y = y0 + y1;
                if constexpr (FP32) y *= spow[n1];
                YZ[it] = y;
            }
            group_sync(bar, GS);
            // d/dA and d/dP per bra component pair
            for (int ab = lane; ab < NAB; ab += GS) {
                const int ma = ab / NB, mb = ab % NB;
                int ax, ay, bx, by;
                {
                    int c = ma, q = 0;
                    while ((q + 1) * (q + 2) / 2 <= c) ++q;
                    ay = q - (c - q * (q + 1) / 2);
                    ax = LA - q;
                    c = mb;
                    q = 0;
                    while ((q + 1) * (q + 2) / 2 <= c) ++q;
                    by = q - (c - q * (q + 1) / 2);
                    bx = LB - q;
                }
                const int az = LA - ax - ay, bz = LB - bx - by;
                const F za2 = (F)(2.0 * pp.za[ip]);
                const F *y = YZ + ab * NH1P;
                const F *Ex = Eb, *Ey = Eb + Lay::NEB, *Ez = Eb + 2 * Lay::NEB;
                const int nx = ax + bx, ny = ay + by, nz = az + bz;
                F a0 = 0, a1 = 0, a2 = 0, t0 = 0, t1 = 0, t2 = 0;
                for (int t = 0; t <= nx + 1; ++t) {
                    const F ex = t <= nx ? Ex[ebi(ax, bx, t, BJ, BT)] : F(0);
                    const F dxv = za2 * Ex[ebi(ax + 1, bx, t, BJ, BT)] - (ax > 0 ? F(ax) * Ex[ebi(ax - 1, bx, t, BJ, BT)] : F(0));
                    for (int u = 0; u <= ny + 1; ++u) {
                        const F ey = u <= ny ? Ey[ebi(ay, by, u, BJ, BT)] : F(0);
                        const F dyv = za2 * Ey[ebi(ay + 1, by, u, BJ, BT)] - (ay > 0 ? F(ay) * Ey[ebi(ay - 1, by, u, BJ, BT)] : F(0));
                        for (int v = 0; v <= nz + 1; ++v) {
                            if (t + u + v > L1 + 1) continue;
                            const F ez = v <= nz ? Ez[ebi(az, bz, v, BJ, BT)] : F(0);
                            const F dzv = za2 * Ez[ebi(az + 1, bz, v, BJ, BT)] - (az > 0 ? F(az) * Ez[ebi(az - 1, bz, v, BJ, BT)] : F(0));
                            const F yy = y[hidx(t, u, v)];
                            if (u <= ny && v <= nz) a0 += dxv * ey * ez * yy;
                            if (t <= nx && v <= nz) a1 += ex * dyv * ez * yy;
                            if (t <= nx && u <= ny) a2 += ex * ey * dzv * yy;
                            if (t <= nx && u <= ny && v <= nz) {
                                const F e3 = ex * ey * ez;
                                t0 += e3 * y[hidx(t + 1, u, v)];
                                t1 += e3 * y[hidx(t, u + 1, v)];
                                t2 += e3 * y[hidx(t, u, v + 1)];
                            }
                        }
                    }
                }
                acc[0] += (double)a0;
                acc[1] += (double)a1;
                acc[2] += (double)a2;
                acc[3] += (double)t0;
                acc[4] += (double)t1;
                acc[5] += (double)t2;
            }
            group_sync(bar, GS);
            // z[cd][h2] = sum_h1 F[cd][h1] s^{|h1|} R[h1+h2] (+ lr), times (-1)^{|h2|} s^{|h2|}
            for (int it = lane; it < NCD * NH2P; it += GS) {
                const int cd = it / NH2P, h2 = it % NH2P;
                int n2 = 0;
                while (nherm(n2) <= h2) ++n2;
                const int r2 = h2 - nherm(n2 - 1);
                int s2 = 0;
                while ((s2 + 1) * (s2 + 2) / 2 <= r2) ++s2;
                const int v2 = r2 - s2 * (s2 + 1) / 2, u2 = s2 - v2, t2 = n2 - s2;
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
                YZ[it] = (n2 & 1) ? -z : z;
            }
            group_sync(bar, GS);
            // d/dC per ket component pair
            for (int cd = lane; cd < NCD; cd += GS) {
                const int mc = cd / ND, md = cd % ND;
                int cx, cy, dx, dy;
                {
                    int c = mc, q = 0;
                    while ((q + 1) * (q + 2) / 2 <= c) ++q;
                    cy = q - (c - q * (q + 1) / 2);
                    cx = LC - q;
                    c = md;
                    q = 0;
                    while ((q + 1) * (q + 2) / 2 <= c) ++q;
                    dy = q - (c - q * (q + 1) / 2);
                    dx = LD - q;
                }
                const int cz = LC - cx - cy, dz = LD - dx - dy;
                const F zc2 = (F)(2.0 * pp.za[kp]);
                const F *z = YZ + cd * NH2P;
                const F *Ex = Ek, *Ey = Ek + Lay::NEK, *Ez = Ek + 2 * Lay::NEK;
                const int nx = cx + dx, ny = cy + dy, nz = cz + dz;
                F c0 = 0, c1 = 0, c2 = 0;
                for (int t = 0; t <= nx + 1; ++t) {
                    const F ex = t <= nx ? Ex[ebi(cx, dx, t, KJ, KT)] : F(0);
                    const F dxv = zc2 * Ex[ebi(cx + 1, dx, t, KJ, KT)] - (cx > 0 ? F(cx) * Ex[ebi(cx - 1, dx, t, KJ, KT)] : F(0));
                    for (int u = 0; u <= ny + 1; ++u) {
                        const F ey = u <= ny ? Ey[ebi(cy, dy, u, KJ, KT)] : F(0);
                        const F dyv = zc2 * Ey[ebi(cy + 1, dy, u, KJ, KT)] - (cy > 0 ? F(cy) * Ey[ebi(cy - 1, dy, u, KJ, KT)] : F(0));
                        for (int v = 0; v <= nz + 1; ++v) {
                            if (t + u + v > L2 + 1) continue;
                            const F ez = v <= nz ? Ez[ebi(cz, dz, v, KJ, KT)] : F(0);
                            const F dzv = zc2 * Ez[ebi(cz + 1, dz, v, KJ, KT)] - (cz > 0 ? F(cz) * Ez[ebi(cz - 1, dz, v, KJ, KT)] : F(0));
                            const F zz = z[hidx(t, u, v)];
                            if (u <= ny && v <= nz) c0 += dxv * ey * ez * zz;
                            if (t <= nx && v <= nz) c1 += ex * dyv * ez * zz;
                            if (t <= nx && u <= ny) c2 += ex * ey * dzv * zz;
                        }
                    }
                }
                acc[6] += (double)c0;
                acc[7] += (double)c1;
                acc[8] += (double)c2;
            }
            group_sync(bar, GS);
        }
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
    unsigned long long nq = 0, npq = 0;
    // unit = (tile, chunk, split): chunk c holds quartets c * QPC ... of the
    // tile, split s takes the bra primitive pairs s, s + S, ...
    const int S = cl.nsplit, C = cl.nchunk, QPC = TILE / C;
    for (long long it = blockIdx.x; it < cl.ntiles * C * S; it += gridDim.x) {
        const long long tile = it / (C * S);
        const int chunk = (int)((it / S) % C), split = (int)(it % S);
        const uint4 tl = cl.tiles[tile];
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
    }
    if ((threadIdx.x & 31) == 0 && (nq || npq)) {  // a split unit may hold primitives only
        atomicAdd(out.counters + 0, nq);
        atomicAdd(out.counters + (sizeof(F) == 4 ? 3 : 1), npq);
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

// Kernel kind per class: the cooperative kernel is compiled for the fp64
// classes with at least 54 function quartets and the fp32 classes with at
// least 648, the thread kernel for every class below 648 (above, its
// per-thread arrays run to tens of KB of local memory).  By default the
// cooperative kernel runs for the fp64 classes from 216 function quartets
// on ((dd|ds) and larger, measured faster there) and wherever it is the
// only one.  ClassLaunch::kind = 1 / 2 forces the
// thread / cooperative kernel where both exist.
template <int LA, int LB, int LC, int LD>
struct UseCoop {
    static constexpr int nfq = ncart(LA) * ncart(LB) * ncart(LC) * ncart(LD);
    static constexpr bool fp64 = nfq >= 54;
    static constexpr bool fp32 = nfq >= 648;
    static constexpr bool thread = nfq < 648;
    static constexpr bool fp64_default = nfq >= 216;
};

template <int LA, int LB, int LC, int LD, typename F>
cudaError_t launch_coop(int gcap, size_t smem, cudaStream_t st, const MolDesc *mols, const ClassLaunch &cl,
                        const OutArgs &out, const double *boys)
{
    using C = CoopChoice<LA, LB, LC, LD, F>;
    return launch_units(k_grad_coop<LA, LB, LC, LD, F, C::GS>, TILE / C::GS, gcap, smem + C::bytes_all(), st, mols,
                        cl, out, boys);
}

template <int LA, int LB, int LC, int LD>
cudaError_t launch_class_kernel(int fp32, int gcap, size_t smem, cudaStream_t st, const MolDesc *mols,
                                const ClassLaunch &cl, const OutArgs &out, const double *boys)
{
    using U = UseCoop<LA, LB, LC, LD>;
    if (fp32) {
        if constexpr (U::fp32) {
            if (!U::thread || cl.kind != 1)
                return launch_coop<LA, LB, LC, LD, float>(gcap, smem, st, mols, cl, out, boys);
        }
    } else {
        if constexpr (U::fp64) {
            if (!U::thread || cl.kind == 2 || (cl.kind == 0 && U::fp64_default))
                return launch_coop<LA, LB, LC, LD, double>(gcap, smem, st, mols, cl, out, boys);
        }
    }
    if constexpr (U::thread) return launch_thread_kernel<LA, LB, LC, LD>(fp32, gcap, smem, st, mols, cl, out, boys);
    return cudaErrorInvalidValue;  // not reached: classes without a thread kernel return above
}

}  // namespace tg
