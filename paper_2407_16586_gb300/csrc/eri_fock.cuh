// Fock-type build (Sec. II.B, the two-electron part of eqs. G_2e and zfock):
// one warp per canonical shell quartet, as the warp gradient kernel.
//
// The density pairs are combined beforehand (the result is linear in them)
// into S_J = sum_p c_J (B_p + B_p^T), B_K = sum_p c_K B_p and B_lr =
// sum_p c_K_lr B_p.  Per canonical quartet (a b|c d) with integrals
// I_s(m n|l s) of both operators s (McMurchie-Davidson, W form over the
// ket primitive pairs and index boxes, as in eri_warp.cuh, without
// derivatives), the 8 permutation images of every integral give
//   Coulomb:  F[m][n], F[n][m] += I_0 S_J[l][s];   F[l][s], F[s][l] += I_0 S_J[m][n]
//   exchange: F[m][l] += I.B[n][s]   F[n][l] += I.B[m][s]   F[m][s] += I.B[n][l]
//             F[n][s] += I.B[m][l]   F[l][m] += I.B[s][n]   F[s][m] += I.B[l][n]
//             F[l][n] += I.B[s][m]   F[s][n] += I.B[l][m]
// with I.B = I_0 B_K + I_1 B_lr, all times 1/|stabiliser| of the quartet.
// Each target block is summed over the quartet on the warp and added to F
// with fp64 atomics.
#pragma once
#include "eri_warp.cuh"

namespace tg {

template <int LA, int LB, int LC, int LD>
struct FockLayout {
    static constexpr int NA = ncart(LA), NB = ncart(LB), NC = ncart(LC), ND = ncart(LD);
    static constexpr int NAB = NA * NB, NCD = NC * ND;
    static constexpr int L1 = LA + LB, L2 = LC + LD, L = L1 + L2;
    static constexpr int NH1 = nherm(L1), NH2 = nherm(L2), NR = nherm(L);
    static constexpr int BJ = LB + 1, BT = L1 + 2, KJ = LD + 1, KT = L2 + 2;
    static constexpr int EBN = (LA + 2) * BJ * BT;  // pair_table layout (one row beyond what the build needs)
    static constexpr int EKN = (LC + 2) * KJ * KT;
    static constexpr int SC_X = 0, SC_T = 3, SC_TH2 = 4, SC_PW = 5;
    static constexpr int NSC = SC_PW + 2 * (L + 1);
    static constexpr int QT_RAW = (int)((6144 / sizeof(double)) / (3 * EKN + NSC));
    static constexpr int QT = QT_RAW < 4 ? 4 : (QT_RAW > 32 ? 32 : QT_RAW);
    static constexpr int KW = (NCD * NH1 + 31) / 32;
    static constexpr int o_I = 0;                       // [2][NAB][NCD]
    static constexpr int o_W = o_I + 2 * NAB * NCD;     // [2][NCD][NH1]
    static constexpr int o_E3b = o_W + 2 * NCD * NH1;   // [NAB][NH1]
    static constexpr int o_E3k = o_E3b + NAB * NH1;     // [NCD][NH2]
    static constexpr int o_R = o_E3k + NCD * NH2;       // [2][NR]
    static constexpr int o_base = o_R + 2 * NR;         // [2][L+1]
    static constexpr int o_Eb = o_base + 2 * (L + 1);   // [3][EBN]
    static constexpr int o_Ek = o_Eb + 3 * EBN;         // [QT][3][EKN]
    static constexpr int o_sc = o_Ek + QT * 3 * EKN;    // [QT][NSC]
    static constexpr int TOTAL = o_sc + QT * NSC;
    static constexpr size_t BYTES = (sizeof(double) * (size_t)TOTAL + 15) & ~(size_t)15;
};

// Per-quartet Fock bound: 8 Q_ab Q_cd M_q (see tg_fock2e in tdgrad.h).
__device__ __forceinline__ bool keep_quartet_fock(const ScreenArgs &scr, const PairSet &bra, const PairSet &ket,
                                                  int bi, int ki, int sa, int sb, int sc, int sd)
{
    if (scr.tau > 0.0) {
        const int ns = scr.nshell;
        const double *M = scr.M;
        double Mq = M[(size_t)sa * ns + sb];
        Mq = fmax(Mq, M[(size_t)sc * ns + sd]);
        Mq = fmax(Mq, M[(size_t)sa * ns + sc]);
        Mq = fmax(Mq, M[(size_t)sa * ns + sd]);
        Mq = fmax(Mq, M[(size_t)sb * ns + sc]);
        Mq = fmax(Mq, M[(size_t)sb * ns + sd]);
        if (scr.scale * bra.Q[bi] * ket.Q[ki] * Mq < scr.tau) return false;
    }
    return true;
}

// Integrals of one canonical quartet (both operators) into I[2][NAB][NCD].
template <int LA, int LB, int LC, int LD>
__device__ void quartet_fock_ints(double *sm, int lane, const GeoArgs &geo, const PrimPairs &pp, int nops,
                                  double omega, int sa, int sb, int sc, int sd, int pb0, int nbp, int ib0, int ibs,
                                  int pk0, int nkp, const double *boys)
{
    using Lay = FockLayout<LA, LB, LC, LD>;
    constexpr int NB = Lay::NB, ND = Lay::ND, NAB = Lay::NAB, NCD = Lay::NCD;
    constexpr int L = Lay::L, NH1 = Lay::NH1, NH2 = Lay::NH2, NR = Lay::NR;
    constexpr int BJ = Lay::BJ, BT = Lay::BT, KJ = Lay::KJ, KT = Lay::KT, EBN = Lay::EBN, EKN = Lay::EKN;
    constexpr int QT = Lay::QT, NSC = Lay::NSC, KW = Lay::KW;
    double *I = sm + Lay::o_I, *W = sm + Lay::o_W, *E3b = sm + Lay::o_E3b, *E3k = sm + Lay::o_E3k;
    double *R = sm + Lay::o_R, *base = sm + Lay::o_base, *Eb = sm + Lay::o_Eb, *Ekall = sm + Lay::o_Ek;
    double *scall = sm + Lay::o_sc;
    const double om2 = omega * omega;
    const bool ominf = isinf(omega);
    const double *xa = geo.xyz + 3 * geo.sh_atom[sa], *xb = geo.xyz + 3 * geo.sh_atom[sb];
    const double *xc = geo.xyz + 3 * geo.sh_atom[sc], *xd = geo.xyz + 3 * geo.sh_atom[sd];
    for (int it = lane; it < 2 * NAB * NCD; it += 32) I[it] = 0.0;
    const bool ket_once = nkp <= QT;
    if (ket_once)
        for (int it = lane; it < 3 * nkp; it += 32) {
            const int j = it / 3, dir = it % 3;
            pair_table<LC, LD, double>(Ekall + (j * 3 + dir) * EKN, pp, pk0 + j, dir, xc[dir], xd[dir]);
        }
    __syncwarp();
    for (int ib = ib0; ib < nbp; ib += ibs) {
        const int ip = pb0 + ib;
        if (lane < 3) pair_table<LA, LB, double>(Eb + lane * EBN, pp, ip, lane, xa[lane], xb[lane]);
        __syncwarp();
        for (int it = lane; it < NAB * NH1; it += 32) {
            const int ab = it / NH1, h = it % NH1;
            int t, u, v, ax, ay, az, bx, by, bz;
            herm_tuv(h, t, u, v);
            cart_xyz(LA, ab / NB, ax, ay, az);
            cart_xyz(LB, ab % NB, bx, by, bz);
            double e = 0.0;
            if (t <= ax + bx && u <= ay + by && v <= az + bz)
                e = Eb[(ax * BJ + bx) * BT + t] * Eb[EBN + (ay * BJ + by) * BT + u] *
                    Eb[2 * EBN + (az * BJ + bz) * BT + v];
            E3b[it] = e;
        }
        double w0r[KW], w1r[KW];
#pragma unroll
        for (int k = 0; k < KW; ++k) w0r[k] = w1r[k] = 0.0;
        for (int q0 = 0; q0 < nkp; q0 += QT) {
            const int nq = min(QT, nkp - q0);
            if (!ket_once)
                for (int it = lane; it < 3 * nq; it += 32) {
                    const int j = it / 3, dir = it % 3;
                    pair_table<LC, LD, double>(Ekall + (j * 3 + dir) * EKN, pp, pk0 + q0 + j, dir, xc[dir], xd[dir]);
                }
            if (lane < nq) {
                double *sc_ = scall + lane * NSC;
                const int kp = pk0 + q0 + lane;
                const double p = pp.p[ip], q = pp.p[kp], pq = p + q, rho = p * q / pq;
                const double X = pp.Px[ip] - pp.Px[kp], Y = pp.Py[ip] - pp.Py[kp], Z = pp.Pz[ip] - pp.Pz[kp];
                const double th2 = (nops == 2) ? (ominf ? 1.0 : om2 / (om2 + rho)) : 1.0;
                const double pref = 34.986836655249725 / (p * q * sqrt(pq)) * pp.K[ip] * pp.K[kp];
                sc_[0] = X;
                sc_[1] = Y;
                sc_[2] = Z;
                sc_[Lay::SC_T] = rho * (X * X + Y * Y + Z * Z);
                sc_[Lay::SC_TH2] = th2;
                double b0 = pref, b1 = pref * sqrt(th2);
                const double m0 = -2.0 * rho, m1 = -2.0 * rho * th2;
#pragma unroll
                for (int m = 0; m <= L; ++m) {
                    sc_[Lay::SC_PW + m] = b0;
                    sc_[Lay::SC_PW + L + 1 + m] = b1;
                    b0 *= m0;
                    b1 *= m1;
                }
            }
            __syncwarp();
            for (int j = 0; j < nq; ++j) {
                const double *sc_ = scall + j * NSC;
                const double *Ek = Ekall + (ket_once ? (q0 + j) : j) * 3 * EKN;
                {
                    const int op = lane >> 4, m = lane & 15;
                    if (op < nops && m <= L) {
                        const double T = sc_[Lay::SC_T] * (op ? sc_[Lay::SC_TH2] : 1.0);
                        base[op * (L + 1) + m] = sc_[Lay::SC_PW + op * (L + 1) + m] * boys_order_fp64(T, m, boys);
                    }
                }
                __syncwarp();
                {
                    const double X = sc_[0], Y = sc_[1], Z = sc_[2];
                    if (lane < nops) R[lane * NR] = base[lane * (L + 1) + L];
                    __syncwarp();
#pragma unroll 1
                    for (int n = L - 1; n >= 0; --n) {
                        const int ne = nherm(L - n) - 1;
                        const int items = nops * ne;
#pragma unroll 1
                        for (int i0 = 0; i0 < items; i0 += 32) {
                            const int it = i0 + lane;
                            double val = 0.0;
                            int dst = -1;
                            if (it < items) {
                                const int op = it / ne, idx = ne - it % ne;
                                int t, u, v;
                                herm_tuv(idx, t, u, v);
                                const double *c = R + op * NR;
                                if (t > 0) {
                                    val = X * c[hidx(t - 1, u, v)];
                                    if (t > 1) val += double(t - 1) * c[hidx(t - 2, u, v)];
                                } else if (u > 0) {
                                    val = Y * c[hidx(t, u - 1, v)];
                                    if (u > 1) val += double(u - 1) * c[hidx(t, u - 2, v)];
                                } else {
                                    val = Z * c[hidx(t, u, v - 1)];
                                    if (v > 1) val += double(v - 1) * c[hidx(t, u, v - 2)];
                                }
                                dst = op * NR + idx;
                            }
                            __syncwarp();
                            if (dst >= 0) R[dst] = val;
                            __syncwarp();
                        }
                        if (lane < nops) R[lane * NR] = base[lane * (L + 1) + n];
                        __syncwarp();
                    }
                }
                for (int it = lane; it < NCD * NH2; it += 32) {
                    const int cd = it / NH2, h = it % NH2;
                    int t, u, v, cx, cy, cz, dx, dy, dz;
                    herm_tuv(h, t, u, v);
                    cart_xyz(LC, cd / ND, cx, cy, cz);
                    cart_xyz(LD, cd % ND, dx, dy, dz);
                    double e = 0.0;
                    if (t <= cx + dx && u <= cy + dy && v <= cz + dz) {
                        e = Ek[(cx * KJ + dx) * KT + t] * Ek[EKN + (cy * KJ + dy) * KT + u] *
                            Ek[2 * EKN + (cz * KJ + dz) * KT + v];
                        e = flip_if(e, t + u + v);
                    }
                    E3k[it] = e;
                }
                __syncwarp();
                const double *R0 = R, *R1 = R + NR;
#pragma unroll
                for (int k = 0; k < KW; ++k) {
                    const int it = lane + 32 * k;
                    if (it >= NCD * NH1) break;
                    const int cd = it / NH1, h1 = it % NH1;
                    int t1, u1, v1, cx, cy, cz, dx, dy, dz;
                    herm_tuv(h1, t1, u1, v1);
                    cart_xyz(LC, cd / ND, cx, cy, cz);
                    cart_xyz(LD, cd % ND, dx, dy, dz);
                    const int nx = cx + dx, ny = cy + dy, nz = cz + dz;
                    const double *e = E3k + cd * NH2;
                    double a0 = 0.0, a1 = 0.0;
                    for (int t2 = 0; t2 <= nx; ++t2)
                        for (int u2 = 0; u2 <= ny; ++u2)
                            for (int v2 = 0; v2 <= nz; ++v2) {
                                const double ev = e[hidx(t2, u2, v2)];
                                const int r = hidx(t1 + t2, u1 + u2, v1 + v2);
                                a0 += ev * R0[r];
                                a1 += ev * R1[r];
                            }
                    w0r[k] += a0;
                    w1r[k] += a1;
                }
                __syncwarp();
            }
        }
#pragma unroll
        for (int k = 0; k < KW; ++k) {
            const int it = lane + 32 * k;
            if (it < NCD * NH1) {
                W[it] = w0r[k];
                W[NCD * NH1 + it] = w1r[k];
            }
        }
        __syncwarp();
        // I_s[ab][cd] += sum_{h1 in box(ab)} E^{ab}_{h1} W_s[cd][h1]
        for (int it = lane; it < NAB * NCD; it += 32) {
            const int ab = it / NCD, cd = it % NCD;
            int ax, ay, az, bx, by, bz;
            cart_xyz(LA, ab / NB, ax, ay, az);
            cart_xyz(LB, ab % NB, bx, by, bz);
            const int nx = ax + bx, ny = ay + by, nz = az + bz;
            const double *e = E3b + ab * NH1, *w0 = W + cd * NH1, *w1 = W + NCD * NH1 + cd * NH1;
            double i0 = 0.0, i1 = 0.0;
            for (int t = 0; t <= nx; ++t)
                for (int u = 0; u <= ny; ++u)
                    for (int v = 0; v <= nz; ++v) {
                        const int h = hidx(t, u, v);
                        i0 += e[h] * w0[h];
                        i1 += e[h] * w1[h];
                    }
            I[it] += i0;
            I[NAB * NCD + it] += i1;
        }
        __syncwarp();
    }
}

// Contractions of I with the density images and the atomic adds to F.
template <int LA, int LB, int LC, int LD>
__device__ void quartet_fock_scatter(const double *I, int lane, int nops, const double *SJ, const double *BK,
                                     const double *BL, int nbf, int fa, int fb, int fc, int fd, double scale,
                                     double *F)
{
    using Lay = FockLayout<LA, LB, LC, LD>;
    constexpr int NA = Lay::NA, NB = Lay::NB, NC = Lay::NC, ND = Lay::ND, NCD = Lay::NCD, NAB = Lay::NAB;
    const double *I1 = I + NAB * NCD;
    auto ix = [&](int ia, int ib, int ic, int id) { return (ia * NB + ib) * NCD + ic * ND + id; };
    // Coulomb: F[m][n], F[n][m] += sum_{ls} I0 S_J[l][s]
    for (int it = lane; it < NAB; it += 32) {
        const int ia = it / NB, ib = it % NB;
        double acc = 0.0;
        for (int ic = 0; ic < NC; ++ic)
            for (int id = 0; id < ND; ++id) acc += I[ix(ia, ib, ic, id)] * SJ[(size_t)(fc + ic) * nbf + fd + id];
        acc *= scale;
        atomicAdd(F + (size_t)(fa + ia) * nbf + fb + ib, acc);
        atomicAdd(F + (size_t)(fb + ib) * nbf + fa + ia, acc);
    }
    // Coulomb: F[l][s], F[s][l] += sum_{mn} I0 S_J[m][n]
    for (int it = lane; it < NCD; it += 32) {
        const int ic = it / ND, id = it % ND;
        double acc = 0.0;
        for (int ia = 0; ia < NA; ++ia)
            for (int ib = 0; ib < NB; ++ib) acc += I[ix(ia, ib, ic, id)] * SJ[(size_t)(fa + ia) * nbf + fb + ib];
        acc *= scale;
        atomicAdd(F + (size_t)(fc + ic) * nbf + fd + id, acc);
        atomicAdd(F + (size_t)(fd + id) * nbf + fc + ic, acc);
    }
    // exchange: eight images, target (row index, column index) and summed
    // indices; shell offsets by position 0..3 = a, b, c, d
    const int off[4] = {fa, fb, fc, fd};
    const int nn[4] = {NA, NB, NC, ND};
    // image k: target F[x][y] += sum I(m n|l s) B[u][v]; positions (x, y, u, v)
    const int img[8][4] = {{0, 2, 1, 3}, {1, 2, 0, 3}, {0, 3, 1, 2}, {1, 3, 0, 2},
                           {2, 0, 3, 1}, {3, 0, 2, 1}, {2, 1, 3, 0}, {3, 1, 2, 0}};
#pragma unroll 1
    for (int k = 0; k < 8; ++k) {
        const int X = img[k][0], Y = img[k][1], U = img[k][2], V = img[k][3];
        const int nx = nn[X], ny = nn[Y], nu = nn[U], nv = nn[V];
        for (int it = lane; it < nx * ny; it += 32) {
            int pos[4];
            pos[X] = it / ny;
            pos[Y] = it % ny;
            double acc = 0.0;
            for (int u = 0; u < nu; ++u)
                for (int v = 0; v < nv; ++v) {
                    pos[U] = u;
                    pos[V] = v;
                    const int e = ix(pos[0], pos[1], pos[2], pos[3]);
                    const size_t bi = (size_t)(off[U] + u) * nbf + off[V] + v;
                    acc += I[e] * BK[bi];
                    if (nops == 2) acc += I1[e] * BL[bi];
                }
            atomicAdd(F + (size_t)(off[X] + pos[X]) * nbf + off[Y] + pos[Y], acc * scale);
        }
    }
}

// Persistent Fock class kernel over tile units (as k_grad_warp).  The
// combined matrices are den.A[0] = S_J, den.B[0] = B_K, den.A[1] = B_lr.
template <int LA, int LB, int LC, int LD>
__global__ void __launch_bounds__(TILE, 2) k_fock_warp(const MolDesc *__restrict__ mols, ClassLaunch cl, OutArgs out,
                                                       const double *__restrict__ boys)
{
    using Lay = FockLayout<LA, LB, LC, LD>;
    const int NG = blockDim.x / 32;
    extern __shared__ double smem[];
    const int grp = threadIdx.x / 32, lane = threadIdx.x % 32;
    double *wsm = smem + (size_t)grp * (Lay::BYTES / sizeof(double));
    unsigned long long nq = 0, npq = 0, nbv = 0;
    const int S = cl.nsplit, C = cl.nchunk, QPC = TILE / C;
    for (long long it = blockIdx.x; it < cl.ntiles * C * S; it += gridDim.x) {
        const long long tile = it / (C * S);
        const int chunk = (int)((it / S) % C), split = (int)(it % S);
        const uint4 tl = cl.tiles[tile * cl.stride];
        const MolDesc &md = mols[tl.x];
        const PairSet bra = md.sets[cl.P], ket = md.sets[cl.Q];
        const bool same = cl.P == cl.Q;
        for (int qi = chunk * QPC + grp; qi < (chunk + 1) * QPC; qi += NG) {
            const int bi = tl.y * TB + qi / TK;
            const int ki = tl.z * TK + qi % TK;
            bool ok = bi < bra.n && ki < ket.n && (!same || bi >= ki);
            if (ok) ok = split < bra.np[bi];
            int sa = 0, sb = 0, sc = 0, sd = 0;
            if (ok) {
                sa = bra.sa[bi];
                sb = bra.sb[bi];
                sc = ket.sa[ki];
                sd = ket.sb[ki];
                ok = keep_quartet_fock(md.scr, bra, ket, bi, ki, sa, sb, sc, sd);
            }
            if (!ok) continue;  // uniform across the warp
            double scale = 1.0;
            if (sa == sb) scale *= 0.5;
            if (sc == sd) scale *= 0.5;
            if (same && bi == ki) scale *= 0.5;
            const int nbp = bra.np[bi], nkp = ket.np[ki];
            const int nops = md.den.use_lr ? 2 : 1;
            quartet_fock_ints<LA, LB, LC, LD>(wsm, lane, md.geo, md.pp, nops, md.den.omega, sa, sb, sc, sd,
                                              bra.poff[bi], nbp, split, S, ket.poff[ki], nkp, boys);
            const int *bf = md.geo.sh_bf;
            quartet_fock_scatter<LA, LB, LC, LD>(wsm + Lay::o_I, lane, nops, md.den.A[0], md.den.B[0], md.den.A[1],
                                                 md.den.nbf, bf[sa], bf[sb], bf[sc], bf[sd], scale, out.fock);
            __syncwarp();
            if (lane == 0) {
                if (split == 0) nq += 1;
                npq += (unsigned long long)((nbp - split + S - 1) / S) * nkp;
                nbv += (unsigned long long)((nbp - split + S - 1) / S);
            }
        }
    }
    if (lane == 0 && (nq || npq)) {
        atomicAdd(out.counters + 0, nq);
        atomicAdd(out.counters + 1, npq);
        atomicAdd(out.counters + 4, nbv);
    }
}

// Warps per CTA: four, or two where four warps' arrays would pass 200 KB ((dd|dd)).
template <int LA, int LB, int LC, int LD>
constexpr int fock_warps()
{
    return 4 * FockLayout<LA, LB, LC, LD>::BYTES <= 200 * 1024 ? 4 : 2;
}

template <int LA, int LB, int LC, int LD>
cudaError_t launch_fock_class(int gcap, cudaStream_t st, const MolDesc *mols, const ClassLaunch &cl,
                              const OutArgs &out, const double *boys)
{
    constexpr int nw = fock_warps<LA, LB, LC, LD>();
    return launch_units(k_fock_warp<LA, LB, LC, LD>, nw, gcap, (size_t)nw * FockLayout<LA, LB, LC, LD>::BYTES, st,
                        mols, cl, out, boys, 32 * nw);
}

}  // namespace tg
