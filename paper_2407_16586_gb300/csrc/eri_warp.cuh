// Warp-cooperative derivative-ERI class kernel: one warp per contracted
// shell quartet, every array in the warp's slice of shared memory, and every
// phase spread over the 32 lanes.
//
// GB300 runs a DFMA warp instruction at the same pipe cost whether one lane
// or all 32 are active, so no phase here is left to a few lanes: the Boys
// function runs one order per lane (Taylor step from the tabulated F_m, no
// recursion), the Hermite R tensors are built level by level with one entry
// per lane, and the contractions are split over (function pair, Hermite
// index) items.  Loops over Hermite indices are restricted to the index box
// where a function pair's expansion coefficients can be non-zero
// (t <= a_x + b_x, u <= a_y + b_y, v <= a_z + b_z, eq. cartG), which removes
// the zero terms of the full tetrahedron t + u + v <= L.
//
// Algebra (McMurchie-Davidson, both operators s = 1/r and erf(w r)/r), for a
// bra primitive pair p and its ket primitive pairs q:
//
//   F_s[cd][h1]  = sum_ab Gamma_s[ab][cd] E^{ab}_{h1}(p)                    (per p)
//   W_s[cd][h1] += sum_{h2 in box(cd)} (-1)^|h2| E^{cd}_{h2}(q) R_s[h1+h2]   (over q)
//   z[cd][h2]    = (-1)^|h2| sum_s sum_h1 F_s[cd][h1] R_s[h1+h2]             (per q)
//   d/dC        += sum dE^{cd}_{h2}/dC_i (q) z[cd][h2]                      (eq. deriv)
//   Y[ab][h1]    = sum_s sum_cd Gamma_s[ab][cd] W_s[cd][h1]                  (per p)
//   d/dA        += sum dE^{ab}_{h1}/dA_i Y[ab][h1]
//   d/dA + d/dB += sum E^{ab}_{h1 - 1_i} Y[ab][h1]   (the R-tensor shift)
//
// and d/dB, d/dD follow from translational invariance (eq. ti).  In fp32 the
// scaled Hermite basis R'_h = R_h / s^{|h|}, s = sqrt(2 rho), keeps every
// value in range; the factors s^{|h|} move onto E^{cd}, W, F and z.  The fp32
// route adds each bra primitive pair's contribution to fp64 accumulators.
#pragma once
#include "eri_coop.cuh"

namespace tg {

// (t, u, v) of every compact Hermite index hidx up to total 9, packed t | u << 8 | v << 16.
struct HermTriples {
    unsigned int tuv[nherm(9)];
};
__host__ __device__ constexpr HermTriples make_herm_triples()
{
    HermTriples h{};
    for (int n = 0; n <= 9; ++n)
        for (int t = n; t >= 0; --t)
            for (int u = n - t; u >= 0; --u) {
                const int v = n - t - u;
                h.tuv[hidx(t, u, v)] = (unsigned)t | ((unsigned)u << 8) | ((unsigned)v << 16);
            }
    return h;
}
static __device__ const HermTriples kHermTriples = make_herm_triples();

// v, negated when odd is 1 (a sign-bit flip on the integer pipe)
__device__ __forceinline__ double flip_if(double v, int odd)
{
    return __longlong_as_double(__double_as_longlong(v) ^ ((long long)(odd & 1) << 63));
}
__device__ __forceinline__ float flip_if(float v, int odd)
{
    return __int_as_float(__float_as_int(v) ^ ((odd & 1) << 31));
}

__device__ __forceinline__ void herm_tuv(int h, int &t, int &u, int &v)
{
    const unsigned w = kHermTriples.tuv[h];
    t = (int)(w & 0xff);
    u = (int)((w >> 8) & 0xff);
    v = (int)(w >> 16);
}

// Cartesian exponents of component c of a shell of angular momentum l <= 2
// (lexicographic: xx, xy, xz, yy, yz, zz)
__device__ __forceinline__ void cart_xyz(int l, int c, int &x, int &y, int &z)
{
    const int s = c == 0 ? 0 : (c < 3 ? 1 : 2);
    z = c - s * (s + 1) / 2;
    y = s - z;
    x = l - s;
}

// F_m(T) for one order m <= BOYS_M - BOYS_TAYLOR, with no recursion over m:
// for T < BOYS_TMAX the Taylor step of the tabulated F_m, F_{m+1}, ... about
// the nearest grid point, F_m(T0 - d) = sum_k F_{m+k}(T0) d^k / k!; above,
// F_0 = sqrt(pi / T) / 2 (erfc(6) < 3e-17) and the m upward steps
// F_{k+1} = ((2k + 1) F_k - e^-T) / (2T), stable for large T.
__device__ __forceinline__ double boys_order_fp64(double T, int m, const double *__restrict__ tab)
{
    if (T < BOYS_TMAX) {
        const int i = __double2int_rn(T * (1.0 / BOYS_H));
        const double d = i * BOYS_H - T;
        const double *row = tab + i * (BOYS_M + 1) + m;
        double acc = row[BOYS_TAYLOR];
#pragma unroll
        for (int k = BOYS_TAYLOR - 1; k >= 0; --k) acc = row[k] + acc * (d * (1.0 / (k + 1)));
        return acc;
    }
    const double it = 1.0 / T;
    double f = 0.88622692545275801365 * sqrt(it);
    const double et = exp(-T), h = 0.5 * it;
    for (int k = 0; k < m; ++k) f = ((2 * k + 1) * f - et) * h;
    return f;
}

// The same in fp32, from the fp32 copy of the table that follows the fp64 one.
__device__ __forceinline__ float boys_order_fp32(float T, int m, const double *__restrict__ tab)
{
    if (T < (float)BOYS_TMAX) {
        const float *ftab = reinterpret_cast<const float *>(tab + BOYS_TAB);
        const int i = __float2int_rn(T * (float)(1.0 / BOYS_H));
        const float d = (float)i * (float)BOYS_H - T;
        const float *row = ftab + i * (BOYS_M + 1) + m;
        float acc = row[BOYS_TAYLOR];
#pragma unroll
        for (int k = BOYS_TAYLOR - 1; k >= 0; --k) acc = row[k] + acc * (d * (1.0f / (k + 1)));
        return acc;
    }
    const float it = 1.0f / T;
    float f = 0.88622692545275801365f * sqrtf(it);
    const float et = __expf(-T), h = 0.5f * it;
    for (int k = 0; k < m; ++k) f = ((2 * k + 1) * f - et) * h;
    return f;
}

// Shared memory of a warp-kernel CTA (TILE / 32 warps of base_n + q * per_q
// elements of fsize bytes, the item lists, and the tile staging plus the
// per-CTA gradient slab of a molecule of up to 32 atoms) and the largest
// q <= q0 (at least 4) with which two such CTAs fit in one SM's 228 KB
// (1 KB reserved per CTA); 0 if none does.
constexpr size_t warp_cta_bytes(size_t fsize, int base_n, int per_q, size_t list_bytes, int q)
{
    return (size_t)(TILE / 32) * ((fsize * (size_t)(base_n + q * per_q) + 15) & ~(size_t)15) + list_bytes + 64 +
           (size_t)TILE * 12 * sizeof(double) + (size_t)TILE * 4 * sizeof(int) + 6 * (TB + TK) * sizeof(double) +
           2 * (TB + TK) * sizeof(int) + 3 * 32 * sizeof(double);
}
constexpr int warp_qt_two_ctas(size_t fsize, int base_n, int per_q, size_t list_bytes, int q0)
{
    for (int q = q0; q >= 4; --q)
        if (2 * (warp_cta_bytes(fsize, base_n, per_q, list_bytes, q) + 1024) <= 228 * 1024) return q;
    return 0;
}

template <int LA, int LB, int LC, int LD, typename F>
struct WarpLayout {
    static constexpr int NA = ncart(LA), NB = ncart(LB), NC = ncart(LC), ND = ncart(LD);
    static constexpr int NAB = NA * NB, NCD = NC * ND;
    static constexpr int L1 = LA + LB, L2 = LC + LD, L = L1 + L2;
    static constexpr int NH1 = nherm(L1), NH1P = nherm(L1 + 1), NH2 = nherm(L2), NH2P = nherm(L2 + 1);
    static constexpr int NR = nherm(L + 1);
    static constexpr int BJ = LB + 1, BT = L1 + 2, KJ = LD + 1, KT = L2 + 2;
    static constexpr int EBN = (LA + 2) * BJ * BT;  // one direction of the bra 1-D table
    static constexpr int EKN = (LC + 2) * KJ * KT;
    // per ket primitive pair scalars: X, Y, Z (fp32: times s), T, th2, pref0, pref1,
    // m0, m1 (fp64: -2 rho, -2 rho th2; fp32: -1, -th2), zc2, s, then s^0 .. s^(L+2)
    static constexpr int SC_X = 0, SC_T = 3, SC_TH2 = 4, SC_PREF = 5, SC_MUL = 7, SC_ZC2 = 9, SC_S = 10,
                         SC_POW = 11;
    // then, per operator, the base multipliers pref_op * mul_op^m for m <= L + 1
    static constexpr int SC_PW = SC_POW + L + 3;
    static constexpr int NSC = SC_PW + 2 * (L + 2);
    // ket primitive pairs whose 1-D tables and scalars are kept at a time: a
    // 6 KB budget per warp, lowered (not below 4) where that lets two CTAs
    // share an SM on small molecules
    static constexpr int PER_Q = 3 * EKN + NSC;
    static constexpr int BASE_N = 2 * NAB * NCD + 2 * NCD * NH1 + 2 * NCD * NH1P + NAB * NH1 + NCD * NH2 + 2 * NR +
                                  2 * (L + 2) + 3 * EBN;
    static constexpr int QT_RAW = (int)((6144 / sizeof(F)) / PER_Q);
    static constexpr int QT0 = QT_RAW < 4 ? 4 : (QT_RAW > 32 ? 32 : QT_RAW);
    static constexpr int ZMAX = NCD * NH2P, YMAX = NAB * NH1P;
    static constexpr size_t LIST_BYTES = (sizeof(unsigned) * (size_t)(ZMAX + YMAX) + 15) & ~(size_t)15;
    static constexpr int QT_FIT = warp_qt_two_ctas(sizeof(F), BASE_N, PER_Q, LIST_BYTES, QT0);
    static constexpr int QT = QT_FIT > 0 ? QT_FIT : QT0;
    // element offsets (F units)
    static constexpr int o_gam = 0;                          // [2][NAB][NCD]
    static constexpr int o_F = o_gam + 2 * NAB * NCD;        // [2][NCD][NH1]
    static constexpr int o_W = o_F + 2 * NCD * NH1;          // [2][NCD][NH1P]
    static constexpr int o_E3b = o_W + 2 * NCD * NH1P;       // [NAB][NH1]
    static constexpr int o_E3k = o_E3b + NAB * NH1;          // [NCD][NH2]
    static constexpr int o_R = o_E3k + NCD * NH2;            // [2][NR]
    static constexpr int o_base = o_R + 2 * NR;              // [2][L+2]
    static constexpr int o_Eb = o_base + 2 * (L + 2);        // [3][EBN]
    static constexpr int o_Ek = o_Eb + 3 * EBN;              // [QT][3][EKN]
    static constexpr int o_sc = o_Ek + QT * 3 * EKN;         // [QT][NSC]
    static constexpr int TOTAL = o_sc + QT * NSC;
    static constexpr size_t BYTES = (sizeof(F) * (size_t)TOTAL + 15) & ~(size_t)15;
    static_assert(o_Ek == BASE_N, "BASE_N counts every array ahead of the ket tables");
    // (ZMAX, YMAX, LIST_BYTES above: the CTA-wide lists of the (cd, h2) items of
    // z and the (ab, h1) items of Y that lie in a derivative box, built once per CTA)
    // W items per lane (kept in registers over the ket primitives)
    static constexpr int KW = (NCD * NH1P + 31) / 32;
    __host__ __device__ static constexpr size_t bytes() { return BYTES; }
};

// 1-D Hermite table of one direction of primitive pair ip, written to dst
// as [i][j][t] (i <= LX + 1, j <= LY, t <= LX + LY + 1).
template <int LX, int LY, typename F>
__device__ __forceinline__ void pair_table(F *dst, const PrimPairs &pp, int ip, int dir, double cen0, double cen1)
{
    constexpr int J1 = LY + 1, T1 = LX + LY + 2;
    F E[LX + 2][LY + 1][LX + LY + 2];
    if constexpr (sizeof(F) == 4) {
        etab<LX + 1, LY>(E, pp.fPA[dir * pp.n + ip], pp.fPB[dir * pp.n + ip], 0.5f / pp.fp[ip]);
    } else {
        const double P = dir == 0 ? pp.Px[ip] : (dir == 1 ? pp.Py[ip] : pp.Pz[ip]);
        etab<LX + 1, LY>(E, (F)(P - cen0), (F)(P - cen1), (F)(0.5 / pp.p[ip]));
    }
#pragma unroll
    for (int i = 0; i <= LX + 1; ++i)
#pragma unroll
        for (int j = 0; j <= LY; ++j)
#pragma unroll
            for (int t = 0; t <= LX + LY + 1; ++t) dst[(i * J1 + j) * T1 + t] = E[i][j][t];
}

// One contracted quartet by one warp, bra primitive pairs ib0, ib0 + ibs, ...
// acc[0..2] += d/dA, acc[3..5] += d/dA + d/dB, acc[6..8] += d/dC (this lane's
// share; the caller sums the warp).
template <int LA, int LB, int LC, int LD, typename F>
__device__ void quartet_warp(F *sm, int lane, const F *smallf, const unsigned *zlist, int nz, const unsigned *ylist, int ny,
                             const GeoArgs &geo, const DensArgs &den, const PrimPairs &pp, int sa, int sb, int sc,
                             int sd, int pb0, int nbp, int ib0, int ibs, int pk0, int nkp, double scale,
                             const double *boys, double (&acc)[9])
{
    using Lay = WarpLayout<LA, LB, LC, LD, F>;
    constexpr int NB = Lay::NB, ND = Lay::ND, NAB = Lay::NAB, NCD = Lay::NCD;
    constexpr int L1 = Lay::L1, L = Lay::L;
    constexpr int NH1 = Lay::NH1, NH1P = Lay::NH1P, NH2 = Lay::NH2, NH2P = Lay::NH2P, NR = Lay::NR;
    constexpr int BJ = Lay::BJ, BT = Lay::BT, KJ = Lay::KJ, KT = Lay::KT, EBN = Lay::EBN, EKN = Lay::EKN;
    constexpr int QT = Lay::QT, NSC = Lay::NSC, KW = Lay::KW;
    constexpr bool FP32 = sizeof(F) == 4;
    F *gam = sm + Lay::o_gam, *Fr = sm + Lay::o_F, *W = sm + Lay::o_W, *E3b = sm + Lay::o_E3b;
    F *E3k = sm + Lay::o_E3k, *R = sm + Lay::o_R, *base = sm + Lay::o_base, *Eb = sm + Lay::o_Eb;
    F *Ekall = sm + Lay::o_Ek, *scall = sm + Lay::o_sc;
    const int nops = den.use_lr ? 2 : 1;
    const double om2 = den.omega * den.omega;
    const bool ominf = isinf(den.omega);
    const int nbf = den.nbf;
    const int fa = geo.sh_bf[sa], fb = geo.sh_bf[sb], fc = geo.sh_bf[sc], fd = geo.sh_bf[sd];
    const double *xa = geo.xyz + 3 * geo.sh_atom[sa], *xb = geo.xyz + 3 * geo.sh_atom[sb];
    const double *xc = geo.xyz + 3 * geo.sh_atom[sc], *xd = geo.xyz + 3 * geo.sh_atom[sd];

    // ---- Gamma_s[ab][cd]: the 8 permutation images of the pair products, times scale
    for (int it = lane; it < NAB * NCD; it += 32) {
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
        gam[NAB * NCD + it] = (F)g1;
    }
    // with one operator the second R tensor stays zero (the sums over both operators read it)
    if (nops == 1)
        for (int it = lane; it < NR; it += 32) R[NR + it] = F(0);
    // ket 1-D tables of the first QT ket primitive pairs (kept for every bra primitive)
    const bool ket_once = nkp <= QT;
    if (ket_once)
        for (int it = lane; it < 3 * nkp; it += 32) {
            const int j = it / 3, dir = it % 3;
            pair_table<LC, LD, F>(Ekall + (j * 3 + dir) * EKN, pp, pk0 + j, dir, xc[dir], xd[dir]);
        }
    __syncwarp();

    for (int ib = ib0; ib < nbp; ib += ibs) {
        const int ip = pb0 + ib;
        // ---- bra tables (lanes 0-2), then E3b[ab][h1] and W = 0
        if (lane < 3) pair_table<LA, LB, F>(Eb + lane * EBN, pp, ip, lane, xa[lane], xb[lane]);
        __syncwarp();
        for (int it = lane; it < NAB * NH1; it += 32) {
            const int ab = it / NH1, h = it % NH1;
            int t, u, v, ax, ay, az, bx, by, bz;
            herm_tuv(h, t, u, v);
            cart_xyz(LA, ab / NB, ax, ay, az);
            cart_xyz(LB, ab % NB, bx, by, bz);
            F e = F(0);
            if (t <= ax + bx && u <= ay + by && v <= az + bz)
                e = Eb[(ax * BJ + bx) * BT + t] * Eb[EBN + (ay * BJ + by) * BT + u] *
                    Eb[2 * EBN + (az * BJ + bz) * BT + v];
            E3b[it] = e;
        }
        __syncwarp();
        // ---- F_s[cd][h1] = sum_ab Gamma_s[ab][cd] E3b[ab][h1]
        for (int it = lane; it < NCD * NH1; it += 32) {
            const int cd = it / NH1, h = it % NH1;
            F s0 = F(0), s1 = F(0);
#pragma unroll 6
            for (int ab = 0; ab < NAB; ++ab) {
                const F e = E3b[ab * NH1 + h];
                s0 += gam[ab * NCD + cd] * e;
                s1 += gam[NAB * NCD + ab * NCD + cd] * e;
            }
            Fr[it] = s0;
            Fr[NCD * NH1 + it] = s1;
        }
        __syncwarp();

        // per-p fp32 partial sums of this lane (fp64 route: accumulated directly)
        F pC0 = F(0), pC1 = F(0), pC2 = F(0);
        // this lane's W items it = lane + 32 k, both operators, in registers
        F w0r[KW], w1r[KW];
#pragma unroll
        for (int k = 0; k < KW; ++k) w0r[k] = w1r[k] = F(0);
        for (int q0 = 0; q0 < nkp; q0 += QT) {
            const int nq = min(QT, nkp - q0);
            // ---- ket tables (when not kept) and per-q scalars, one lane per q
            if (!ket_once)
                for (int it = lane; it < 3 * nq; it += 32) {
                    const int j = it / 3, dir = it % 3;
                    pair_table<LC, LD, F>(Ekall + (j * 3 + dir) * EKN, pp, pk0 + q0 + j, dir, xc[dir], xd[dir]);
                }
            if (lane < nq) {
                F *sc_ = scall + lane * NSC;
                const int kp = pk0 + q0 + lane;
                if constexpr (FP32) {
                    const long long nr = pp.n;
                    const float pf = pp.fp[ip], qf = pp.fp[kp], pq = pf + qf, rho = pf * qf / pq;
                    const float X = pp.fPA[ip] - pp.fPA[kp] + (float)(xa[0] - xc[0]);
                    const float Y = pp.fPA[nr + ip] - pp.fPA[nr + kp] + (float)(xa[1] - xc[1]);
                    const float Z = pp.fPA[2 * nr + ip] - pp.fPA[2 * nr + kp] + (float)(xa[2] - xc[2]);
                    const float s = sqrtf(2.0f * rho);
                    const float om2f = (float)om2;
                    const float th2 = (nops == 2) ? (ominf ? 1.0f : om2f / (om2f + rho)) : 1.0f;
                    const float pref = 34.986836655249725f * rsqrtf(pq) / (pf * qf) * pp.fK[ip] * pp.fK[kp];
                    sc_[0] = X * s;
                    sc_[1] = Y * s;
                    sc_[2] = Z * s;
                    sc_[Lay::SC_T] = rho * (X * X + Y * Y + Z * Z);
                    sc_[Lay::SC_TH2] = th2;
                    sc_[Lay::SC_PREF] = pref;
                    sc_[Lay::SC_PREF + 1] = pref * sqrtf(th2);
                    sc_[Lay::SC_MUL] = -1.0f;
                    sc_[Lay::SC_MUL + 1] = -th2;
                    sc_[Lay::SC_ZC2] = 2.0f * pp.fza[kp];
                    sc_[Lay::SC_S] = s;
                    float pw = 1.0f;
#pragma unroll
                    for (int k = 0; k <= L + 2; ++k) {
                        sc_[Lay::SC_POW + k] = pw;
                        pw *= s;
                    }
                    float b0 = pref, b1 = pref * sqrtf(th2);
#pragma unroll
                    for (int m = 0; m <= L + 1; ++m) {
                        sc_[Lay::SC_PW + m] = b0;
                        sc_[Lay::SC_PW + L + 2 + m] = b1;
                        b0 = -b0;
                        b1 *= -th2;
                    }
                } else {
                    const double p = pp.p[ip], q = pp.p[kp], pq = p + q, rho = p * q / pq;
                    const double X = pp.Px[ip] - pp.Px[kp], Y = pp.Py[ip] - pp.Py[kp], Z = pp.Pz[ip] - pp.Pz[kp];
                    const double th2 = (nops == 2) ? (ominf ? 1.0 : om2 / (om2 + rho)) : 1.0;
                    const double pref = 34.986836655249725 / (p * q * sqrt(pq)) * pp.K[ip] * pp.K[kp];
                    sc_[0] = X;
                    sc_[1] = Y;
                    sc_[2] = Z;
                    sc_[Lay::SC_T] = rho * (X * X + Y * Y + Z * Z);
                    sc_[Lay::SC_TH2] = th2;
                    sc_[Lay::SC_PREF] = pref;
                    sc_[Lay::SC_PREF + 1] = pref * sqrt(th2);
                    sc_[Lay::SC_MUL] = -2.0 * rho;
                    sc_[Lay::SC_MUL + 1] = -2.0 * rho * th2;
                    sc_[Lay::SC_ZC2] = 2.0 * pp.za[kp];
                    sc_[Lay::SC_S] = 1.0;
#pragma unroll
                    for (int k = 0; k <= L + 2; ++k) sc_[Lay::SC_POW + k] = 1.0;
                    double b0 = pref, b1 = pref * sqrt(th2);
                    const double m0 = -2.0 * rho, m1 = -2.0 * rho * th2;
#pragma unroll
                    for (int m = 0; m <= L + 1; ++m) {
                        sc_[Lay::SC_PW + m] = b0;
                        sc_[Lay::SC_PW + L + 2 + m] = b1;
                        b0 *= m0;
                        b1 *= m1;
                    }
                }
            }
            __syncwarp();

            for (int j = 0; j < nq; ++j) {
                const F *sc_ = scall + j * NSC;
                const F *Ek = Ekall + (ket_once ? (q0 + j) : j) * 3 * EKN;
                // ---- Boys function and R bases: lane (op, m), op = lane / 16
                {
                    const int op = lane >> 4, m = lane & 15;
                    if (op < nops && m <= L + 1) {
                        const F T = sc_[Lay::SC_T] * (op ? sc_[Lay::SC_TH2] : F(1));
                        F fm;
                        if constexpr (FP32) {
                            if (T < 1.0f) {
                                fm = (float)boys_order_fp64((double)T, m, boys);
                            } else {
                                fm = boys_order_fp32(T, m, boys);
                            }
                        } else {
                            fm = boys_order_fp64(T, m, boys);
                        }
                        base[op * (L + 2) + m] = sc_[Lay::SC_PW + op * (L + 2) + m] * fm;
                    }
                }
                __syncwarp();
                // ---- R_s[h] level by level (one entry per lane, in place)
                {
                    const F X = sc_[0], Y = sc_[1], Z = sc_[2];
                    if (lane < nops) R[lane * NR] = base[lane * (L + 2) + L + 1];
                    __syncwarp();
#pragma unroll 1
                    for (int n = L; n >= 0; --n) {
                        const int ne = nherm(L + 1 - n) - 1;  // entries 1 .. ne of this level
                        const int items = nops * ne;
#pragma unroll 1
                        for (int i0 = 0; i0 < items; i0 += 32) {
                            const int it = i0 + lane;
                            F val = F(0);
                            int dst = -1;
                            if (it < items) {
                                const int op = it / ne, idx = ne - it % ne;
                                int t, u, v;
                                herm_tuv(idx, t, u, v);
                                const F *c = R + op * NR;
                                // the integer coefficients come from a table (no int-to-float conversion)
                                if (t > 0) {
                                    val = X * c[hidx(t - 1, u, v)];
                                    if (t > 1) val += smallf[t - 1] * c[hidx(t - 2, u, v)];
                                } else if (u > 0) {
                                    val = Y * c[hidx(t, u - 1, v)];
                                    if (u > 1) val += smallf[u - 1] * c[hidx(t, u - 2, v)];
                                } else {
                                    val = Z * c[hidx(t, u, v - 1)];
                                    if (v > 1) val += smallf[v - 1] * c[hidx(t, u, v - 2)];
                                }
                                dst = op * NR + idx;
                            }
                            __syncwarp();
                            if (dst >= 0) R[dst] = val;
                            __syncwarp();
                        }
                        if (lane < nops) R[lane * NR] = base[lane * (L + 2) + n];
                        __syncwarp();
                    }
                }
                // ---- E3k[cd][h2] = (-1)^|h2| s^|h2| E_x E_y E_z (zero outside the box)
                for (int it = lane; it < NCD * NH2; it += 32) {
                    const int cd = it / NH2, h = it % NH2;
                    int t, u, v, cx, cy, cz, dx, dy, dz;
                    herm_tuv(h, t, u, v);
                    cart_xyz(LC, cd / ND, cx, cy, cz);
                    cart_xyz(LD, cd % ND, dx, dy, dz);
                    F e = F(0);
                    if (t <= cx + dx && u <= cy + dy && v <= cz + dz) {
                        e = Ek[(cx * KJ + dx) * KT + t] * Ek[EKN + (cy * KJ + dy) * KT + u] *
                            Ek[2 * EKN + (cz * KJ + dz) * KT + v];
                        if constexpr (FP32) e *= sc_[Lay::SC_POW + t + u + v];
                        e = flip_if(e, t + u + v);
                    }
                    E3k[it] = e;
                }
                __syncwarp();
                const F *R0 = R, *R1 = R + NR;
                // ---- W_s[cd][h1] += s^|h1| sum_{h2 in box(cd)} E3k[cd][h2] R_s[h1+h2]
#pragma unroll
                for (int k = 0; k < KW; ++k) {
                    const int it = lane + 32 * k;
                    if (it >= NCD * NH1P) break;
                    const int cd = it / NH1P, h1 = it % NH1P;
                    int t1, u1, v1, cx, cy, cz, dx, dy, dz;
                    herm_tuv(h1, t1, u1, v1);
                    cart_xyz(LC, cd / ND, cx, cy, cz);
                    cart_xyz(LD, cd % ND, dx, dy, dz);
                    const int nx = cx + dx, ny = cy + dy, nz = cz + dz;
                    const F *e = E3k + cd * NH2;
                    // fp64: the terms go straight into the lane's W registers;
                    // fp32: the item's sum is scaled by s^|h1| first
                    F w0 = FP32 ? F(0) : w0r[k], w1 = FP32 ? F(0) : w1r[k];
                    for (int t2 = 0; t2 <= nx; ++t2)
                        for (int u2 = 0; u2 <= ny; ++u2)
                            for (int v2 = 0; v2 <= nz; ++v2) {
                                const F ev = e[hidx(t2, u2, v2)];
                                const int r = hidx(t1 + t2, u1 + u2, v1 + v2);
                                w0 += ev * R0[r];
                                w1 += ev * R1[r];
                            }
                    if constexpr (FP32) {
                        const F sh = sc_[Lay::SC_POW + t1 + u1 + v1];
                        w0r[k] += w0 * sh;
                        w1r[k] += w1 * sh;
                    } else {
                        w0r[k] = w0;
                        w1r[k] = w1;
                    }
                }
                // ---- z[cd][h2] over the derivative boxes of cd, contracted with dE^{cd}/dC
                {
                    const F zc2 = sc_[Lay::SC_ZC2];
                    const F *Ex = Ek, *Ey = Ek + EKN, *Ez = Ek + 2 * EKN;
                    F c0 = F(0), c1 = F(0), c2 = F(0);
                    for (int iz = lane; iz < nz; iz += 32) {
                        const unsigned zi = zlist[iz];
                        const int cd = (int)(zi & 0xff), t2 = (int)((zi >> 8) & 0xf), u2 = (int)((zi >> 12) & 0xf),
                                  v2 = (int)((zi >> 16) & 0xf);
                        int cx, cy, cz, dx, dy, dz;
                        cart_xyz(LC, cd / ND, cx, cy, cz);
                        cart_xyz(LD, cd % ND, dx, dy, dz);
                        const int nx = cx + dx, ny = cy + dy, nz = cz + dz;
                        const bool inx = t2 <= nx, iny = u2 <= ny, inz = v2 <= nz;
                        const bool gx = t2 <= nx + 1 && iny && inz, gy = inx && u2 <= ny + 1 && inz,
                                   gz = inx && iny && v2 <= nz + 1;
                        const F *f0 = Fr + cd * NH1, *f1 = Fr + NCD * NH1 + cd * NH1;
                        // both operators in one sum (with one operator, F_1 and R_1 are zero)
                        F z = F(0);
#pragma unroll
                        for (int t1 = 0; t1 <= L1; ++t1)
#pragma unroll
                            for (int u1 = 0; u1 <= L1 - t1; ++u1)
#pragma unroll
                                for (int v1 = 0; v1 <= L1 - t1 - u1; ++v1) {
                                    const int r = hidx(t1 + t2, u1 + u2, v1 + v2);
                                    if constexpr (FP32) {
                                        const F sh = sc_[Lay::SC_POW + t1 + u1 + v1];
                                        z += (f0[hidx(t1, u1, v1)] * R0[r] + f1[hidx(t1, u1, v1)] * R1[r]) * sh;
                                    } else {
                                        z += f0[hidx(t1, u1, v1)] * R0[r];
                                        z += f1[hidx(t1, u1, v1)] * R1[r];
                                    }
                                }
                        const int n2 = t2 + u2 + v2;
                        if constexpr (FP32) z *= sc_[Lay::SC_POW + n2];
                        z = flip_if(z, n2);
                        const F ex = inx ? Ex[(cx * KJ + dx) * KT + t2] : F(0);
                        const F ey = iny ? Ey[(cy * KJ + dy) * KT + u2] : F(0);
                        const F ez = inz ? Ez[(cz * KJ + dz) * KT + v2] : F(0);
                        if (gx) {
                            const F dxv = zc2 * Ex[((cx + 1) * KJ + dx) * KT + t2] -
                                          (cx > 0 && inx ? F(cx) * Ex[((cx - 1) * KJ + dx) * KT + t2] : F(0));
                            c0 += dxv * ey * ez * z;
                        }
                        if (gy) {
                            const F dyv = zc2 * Ey[((cy + 1) * KJ + dy) * KT + u2] -
                                          (cy > 0 && iny ? F(cy) * Ey[((cy - 1) * KJ + dy) * KT + u2] : F(0));
                            c1 += ex * dyv * ez * z;
                        }
                        if (gz) {
                            const F dzv = zc2 * Ez[((cz + 1) * KJ + dz) * KT + v2] -
                                          (cz > 0 && inz ? F(cz) * Ez[((cz - 1) * KJ + dz) * KT + v2] : F(0));
                            c2 += ex * ey * dzv * z;
                        }
                    }
                    pC0 += c0;
                    pC1 += c1;
                    pC2 += c2;
                }
                __syncwarp();  // R, base and E3k are rewritten for the next q
            }
        }
        // ---- W to shared memory for the Y items
#pragma unroll
        for (int k = 0; k < KW; ++k) {
            const int it = lane + 32 * k;
            if (it < NCD * NH1P) {
                W[it] = w0r[k];
                W[NCD * NH1P + it] = w1r[k];
            }
        }
        __syncwarp();
        // ---- Y[ab][h1] = sum_s sum_cd Gamma_s[ab][cd] W_s[cd][h1] with dE/dA and the shifted E
        F a0 = F(0), a1 = F(0), a2 = F(0), t0 = F(0), t1_ = F(0), t2_ = F(0);
        {
            const F za2 = FP32 ? (F)(2.0f * pp.fza[ip]) : (F)(2.0 * pp.za[ip]);
            const F *Ex = Eb, *Ey = Eb + EBN, *Ez = Eb + 2 * EBN;
            for (int iy = lane; iy < ny; iy += 32) {
                const unsigned yi = ylist[iy];
                const int ab = (int)(yi & 0xff), t = (int)((yi >> 8) & 0xf), u = (int)((yi >> 12) & 0xf),
                          v = (int)((yi >> 16) & 0xf), h1 = (int)(yi >> 20);
                int ax, ay, az, bx, by, bz;
                cart_xyz(LA, ab / NB, ax, ay, az);
                cart_xyz(LB, ab % NB, bx, by, bz);
                const int nx = ax + bx, ny = ay + by, nz = az + bz;
                const bool inx = t <= nx, iny = u <= ny, inz = v <= nz;
                const bool gx = t <= nx + 1 && iny && inz, gy = inx && u <= ny + 1 && inz, gz = inx && iny && v <= nz + 1;
                const F *g0 = gam + ab * NCD, *g1 = gam + NAB * NCD + ab * NCD;
                F y = F(0);
#pragma unroll 6
                for (int cd = 0; cd < NCD; ++cd) {
                    y += g0[cd] * W[cd * NH1P + h1];
                    if (nops == 2) y += g1[cd] * W[(NCD + cd) * NH1P + h1];
                }
                const F ex = inx ? Ex[(ax * BJ + bx) * BT + t] : F(0);
                const F ey = iny ? Ey[(ay * BJ + by) * BT + u] : F(0);
                const F ez = inz ? Ez[(az * BJ + bz) * BT + v] : F(0);
                if (gx) {
                    const F dxv = za2 * Ex[((ax + 1) * BJ + bx) * BT + t] -
                                  (ax > 0 && inx ? F(ax) * Ex[((ax - 1) * BJ + bx) * BT + t] : F(0));
                    a0 += dxv * ey * ez * y;
                    if (t >= 1) t0 += Ex[(ax * BJ + bx) * BT + t - 1] * ey * ez * y;
                }
                if (gy) {
                    const F dyv = za2 * Ey[((ay + 1) * BJ + by) * BT + u] -
                                  (ay > 0 && iny ? F(ay) * Ey[((ay - 1) * BJ + by) * BT + u] : F(0));
                    a1 += ex * dyv * ez * y;
                    if (u >= 1) t1_ += ex * Ey[(ay * BJ + by) * BT + u - 1] * ez * y;
                }
                if (gz) {
                    const F dzv = za2 * Ez[((az + 1) * BJ + bz) * BT + v] -
                                  (az > 0 && inz ? F(az) * Ez[((az - 1) * BJ + bz) * BT + v] : F(0));
                    a2 += ex * ey * dzv * y;
                    if (v >= 1) t2_ += ex * ey * Ez[(az * BJ + bz) * BT + v - 1] * y;
                }
            }
        }
        acc[0] += (double)a0;
        acc[1] += (double)a1;
        acc[2] += (double)a2;
        acc[3] += (double)t0;
        acc[4] += (double)t1_;
        acc[5] += (double)t2_;
        acc[6] += (double)pC0;
        acc[7] += (double)pC1;
        acc[8] += (double)pC2;
        __syncwarp();  // E3b, Fr, W and the bra tables are rewritten for the next p
    }
}

// Persistent warp-cooperative class kernel: 4 warps per CTA, warp w takes
// quartets w, w + 4, ... of each unit (tile, chunk, split); the tile's
// 12 x TILE contributions are then added in the same fixed order as k_grad.
template <int LA, int LB, int LC, int LD, typename F>
__global__ void __launch_bounds__(TILE, 2) k_grad_warp(const MolDesc *__restrict__ mols, ClassLaunch cl, OutArgs out,
                                                    const double *__restrict__ boys)
{
    using Lay = WarpLayout<LA, LB, LC, LD, F>;
    constexpr int NG = TILE / 32;
    extern __shared__ double smem[];
    const int nacc3 = out.use_smem ? out.natom_max * 3 : 0;
    double *sg = smem;
    double *stg = smem + nacc3;
    int *sat = reinterpret_cast<int *>(stg + TILE * 12);
    double *tred = reinterpret_cast<double *>(sat + TILE * 4);
    int *ratom = reinterpret_cast<int *>(tred + 6 * (TB + TK));
    unsigned *zlist = reinterpret_cast<unsigned *>(ratom + 2 * (TB + TK));
    unsigned *ylist = zlist + Lay::ZMAX;
    F *wsm = reinterpret_cast<F *>(reinterpret_cast<char *>(zlist) + Lay::LIST_BYTES +
                                   (size_t)(threadIdx.x / 32) * Lay::bytes());
    const int grp = threadIdx.x / 32, lane = threadIdx.x % 32;
    // item lists: (cd, h2) with h2 in a derivative box of cd, (ab, h1) likewise;
    // packed as pair | t << 8 | u << 12 | v << 16 | hermite index << 20
    __shared__ int nlist[2];
    __shared__ F smallf[16];  // 0, 1, ..., 15 as F
    if (threadIdx.x < 16) smallf[threadIdx.x] = F(threadIdx.x);
    if (threadIdx.x == 0) {
        int n = 0;
        for (int cd = 0; cd < Lay::NCD; ++cd)
            for (int h = 0; h < Lay::NH2P; ++h) {
                int t, u, v, cx, cy, cz, dx, dy, dz;
                herm_tuv(h, t, u, v);
                cart_xyz(LC, cd / Lay::ND, cx, cy, cz);
                cart_xyz(LD, cd % Lay::ND, dx, dy, dz);
                const int nx = cx + dx, ny = cy + dy, nz = cz + dz;
                const bool inx = t <= nx, iny = u <= ny, inz = v <= nz;
                if ((t <= nx + 1 && iny && inz) || (inx && u <= ny + 1 && inz) || (inx && iny && v <= nz + 1))
                    zlist[n++] = (unsigned)cd | ((unsigned)t << 8) | ((unsigned)u << 12) | ((unsigned)v << 16) |
                                 ((unsigned)h << 20);
            }
        nlist[0] = n;
        n = 0;
        for (int ab = 0; ab < Lay::NAB; ++ab)
            for (int h = 0; h < Lay::NH1P; ++h) {
                int t, u, v, ax, ay, az, bx, by, bz;
                herm_tuv(h, t, u, v);
                cart_xyz(LA, ab / Lay::NB, ax, ay, az);
                cart_xyz(LB, ab % Lay::NB, bx, by, bz);
                const int nx = ax + bx, ny = ay + by, nz = az + bz;
                const bool inx = t <= nx, iny = u <= ny, inz = v <= nz;
                if ((t <= nx + 1 && iny && inz) || (inx && u <= ny + 1 && inz) || (inx && iny && v <= nz + 1))
                    ylist[n++] = (unsigned)ab | ((unsigned)t << 8) | ((unsigned)u << 12) | ((unsigned)v << 16) |
                                 ((unsigned)h << 20);
            }
        nlist[1] = n;
    }
    __syncthreads();
    const int nz = nlist[0], ny = nlist[1];
    double *slab = out.partials + (size_t)blockIdx.x * out.natom_total * 3;
    int cur = -1, cur_off3 = 0, cur_n3 = 0;
    unsigned long long nq = 0, npq = 0, nbv = 0;
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
            if (ok) {  // uniform across the warp
                double scale = 1.0;
                if (sa == sb) scale *= 0.5;
                if (sc == sd) scale *= 0.5;
                if (same && bi == ki) scale *= 0.5;
                const int nbp = bra.np[bi], nkp = ket.np[ki];
                double acc[9];
#pragma unroll
                for (int k = 0; k < 9; ++k) acc[k] = 0.0;
                quartet_warp<LA, LB, LC, LD, F>(wsm, lane, smallf, zlist, nz, ylist, ny, geo, md.den, pp, sa, sb, sc, sd,
                                                bra.poff[bi], nbp, split, S, ket.poff[ki], nkp, scale, boys, acc);
#pragma unroll
                for (int k = 0; k < 9; ++k)
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], o);
                if (lane == 0) {
#pragma unroll
                    for (int i = 0; i < 3; ++i) {
                        g[i] = acc[i];
                        g[3 + i] = acc[3 + i] - acc[i];
                        g[6 + i] = acc[6 + i];
                        g[9 + i] = -acc[3 + i] - acc[6 + i];
                    }
                    at[0] = geo.sh_atom[sa];
                    at[1] = geo.sh_atom[sb];
                    at[2] = geo.sh_atom[sc];
                    at[3] = geo.sh_atom[sd];
                    if (split == 0) nq += 1;
                    npq += (unsigned long long)((nbp - split + S - 1) / S) * nkp;
                    nbv += (unsigned long long)((nbp - split + S - 1) / S);
                }
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
    if ((threadIdx.x & 31) == 0 && (nq || npq)) {
        atomicAdd(out.counters + 0, nq);
        atomicAdd(out.counters + (sizeof(F) == 4 ? 3 : 1), npq);
        atomicAdd(out.counters + (sizeof(F) == 4 ? 5 : 4), nbv);
        if (sizeof(F) == 4) atomicAdd(out.counters + 2, nq);
    }
}

template <int LA, int LB, int LC, int LD, typename F>
constexpr size_t warp_kernel_smem()
{
    return (size_t)(TILE / 32) * WarpLayout<LA, LB, LC, LD, F>::bytes() + WarpLayout<LA, LB, LC, LD, F>::LIST_BYTES + 64;
}

template <int LA, int LB, int LC, int LD, typename F>
cudaError_t launch_warp(int gcap, size_t smem, cudaStream_t st, const MolDesc *mols, const ClassLaunch &cl,
                        const OutArgs &out, const double *boys)
{
    return launch_units(k_grad_warp<LA, LB, LC, LD, F>, TILE / 32, gcap, smem + warp_kernel_smem<LA, LB, LC, LD, F>(),
                        st, mols, cl, out, boys);
}

// Default class-kernel form per angular class (ssss, psss, psps, ppss, ppps,
// pppp, dsss, dsps, dspp, dsds, dpss, dpps, dppp, dpds, dpdp, ddss, ddps, ddpp,
// ddds, dddp, dddd): 1 = thread, 2 = group, 3 = warp.  Picked from per-class
// kernel times of the mixed route on the 32-atom chain (the fp64 lists there
// hold the largest, most contracted tiles) and of the all-fp64 route; where
// the two disagree by little, the mixed route's choice is kept.
constexpr int kDefaultForm64[NQC] = {1, 1, 1, 1, 1, 3, 1, 1, 1, 3, 1, 3, 3, 3, 3, 3, 3, 3, 3, 2, 2};
constexpr int kDefaultForm32[NQC] = {1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 3, 3, 2, 2};

// Kernel forms per class.  The thread kernel is compiled below 648 function
// quartets (above, its per-thread arrays run to tens of KB of local memory),
// the group kernel for fp64 from 54 and fp32 from 648 function quartets, and
// the warp kernel wherever four warps' arrays fit in shared memory next to
// the tile staging (all classes but (dd|dp) and (dd|dd) in fp64, all but
// (dd|dd) in fp32).  ClassLaunch::kind 1 / 2 / 3 asks for the thread / group /
// warp kernel; a form not compiled for the class falls back to the default.
template <int LA, int LB, int LC, int LD>
struct ClassForms {
    static constexpr int nfq = ncart(LA) * ncart(LB) * ncart(LC) * ncart(LD);
    static constexpr size_t kStageMax = 200 * 1024;  // warp arrays + tile staging (16 KB) per CTA
    static constexpr bool thread = nfq < 648;
    static constexpr bool group64 = nfq >= 54;
    static constexpr bool group32 = nfq >= 648;
    static constexpr bool warp64 = warp_kernel_smem<LA, LB, LC, LD, double>() + 16384 <= kStageMax;
    static constexpr bool warp32 = warp_kernel_smem<LA, LB, LC, LD, float>() + 16384 <= kStageMax;
    // default form per class (1 thread, 2 group, 3 warp): the fastest form
    // measured on GB300 for the 32-atom chain workload, per precision
    static constexpr int qc = pair_class(LA, LB) * (pair_class(LA, LB) + 1) / 2 + pair_class(LC, LD);
    static constexpr int default64 = kDefaultForm64[qc];
    static constexpr int default32 = kDefaultForm32[qc];
    static_assert((default64 != 1 || thread) && (default64 != 2 || group64) && (default64 != 3 || warp64),
                  "default fp64 form not compiled");
    static_assert((default32 != 1 || thread) && (default32 != 2 || group32) && (default32 != 3 || warp32),
                  "default fp32 form not compiled");
};

template <int LA, int LB, int LC, int LD>
cudaError_t launch_class_kernel(int fp32, int gcap, size_t smem, cudaStream_t st, const MolDesc *mols,
                                const ClassLaunch &cl, const OutArgs &out, const double *boys)
{
    using K = ClassForms<LA, LB, LC, LD>;
    int kind = cl.kind;
    if (fp32) {
        if ((kind == 1 && !K::thread) || (kind == 2 && !K::group32) || (kind == 3 && !K::warp32) || kind < 1 || kind > 3)
            kind = K::default32;
        if constexpr (K::warp32)
            if (kind == 3) return launch_warp<LA, LB, LC, LD, float>(gcap, smem, st, mols, cl, out, boys);
        if constexpr (K::group32)
            if (kind == 2) return launch_coop<LA, LB, LC, LD, float>(gcap, smem, st, mols, cl, out, boys);
        if constexpr (K::thread)
            if (kind == 1) return launch_units(k_grad<LA, LB, LC, LD, true>, 0, gcap, smem, st, mols, cl, out, boys);
    } else {
        if ((kind == 1 && !K::thread) || (kind == 2 && !K::group64) || (kind == 3 && !K::warp64) || kind < 1 || kind > 3)
            kind = K::default64;
        if constexpr (K::warp64)
            if (kind == 3) return launch_warp<LA, LB, LC, LD, double>(gcap, smem, st, mols, cl, out, boys);
        if constexpr (K::group64)
            if (kind == 2) return launch_coop<LA, LB, LC, LD, double>(gcap, smem, st, mols, cl, out, boys);
        if constexpr (K::thread)
            if (kind == 1) return launch_units(k_grad<LA, LB, LC, LD, false>, 0, gcap, smem, st, mols, cl, out, boys);
    }
    return cudaErrorInvalidValue;  // not reached: every class compiles its default form
}

}  // namespace tg
