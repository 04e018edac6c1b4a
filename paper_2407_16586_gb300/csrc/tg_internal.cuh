// Internal definitions shared by the tdgrad CUDA translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "tdgrad.h"

namespace tg {

constexpr int MAXL = 2;
constexpr int NPC = 6;   // pair classes (la >= lb): ss ps pp ds dp dd
constexpr int NQC = 21;  // quartet classes (bra pair class >= ket pair class), Sec. II.C
constexpr int TB = 16;   // bra pairs per tile
constexpr int TK = 8;    // ket pairs per tile
constexpr int TILE = TB * TK;
// per-class counters: [0] quartets, [1] fp64 primitive quartets, [2] fp32
// quartets, [3] fp32 primitive quartets, [4] / [5] fp64 / fp32 bra primitive
// pairs visited (one per quartet and bra primitive pair of a unit)
constexpr int NCNT = 6;

// Boys table: F_m(T0) on T0 = 0, 0.05, ..., 36 for m = 0..BOYS_M.
constexpr int BOYS_M = 16;
constexpr int BOYS_NG = 721;
constexpr double BOYS_H = 0.05;
constexpr double BOYS_TMAX = 36.0;
constexpr int BOYS_TAYLOR = 6;
// the fp32 copy of the table follows the fp64 one in the same allocation
constexpr int BOYS_TAB = BOYS_NG * (BOYS_M + 1);

__host__ __device__ constexpr int ncart(int l) { return (l + 1) * (l + 2) / 2; }
// number of Hermite (or Cartesian) triples with total <= L
__host__ __device__ constexpr int nherm(int L) { return L < 0 ? 0 : (L + 1) * (L + 2) * (L + 3) / 6; }
// position of (t,u,v) in the list ordered by total, then t descending, u descending
__host__ __device__ constexpr int hidx(int t, int u, int v)
{
    return nherm(t + u + v - 1) + (u + v) * (u + v + 1) / 2 + v;
}
// component index of (x,y,z) within its shell (lexicographic xx, xy, xz, yy, yz, zz)
__host__ __device__ constexpr int cidx(int x, int y, int z) { return (y + z) * (y + z + 1) / 2 + z; }

__host__ __device__ constexpr int pair_class(int la, int lb) { return la * (la + 1) / 2 + lb; }
__host__ __device__ constexpr int pc_la(int pc) { return pc == 0 ? 0 : (pc <= 2 ? 1 : 2); }
__host__ __device__ constexpr int pc_lb(int pc) { return pc - pair_class(pc_la(pc), 0); }

// Shell pairs of one pair class, sorted by (primitive-pair count, Q') descending.
struct PairSet {
    int n;
    const int *sa, *sb;      // shell indices; l(sa) >= l(sb), equal l: sa >= sb
    const int *poff, *np;    // primitive-pair offset and count
    const double *Q, *Qd;    // Schwarz factors
    const int *key;          // canonical pair key X(X+1)/2 + Y
};

// Primitive pairs (SoA).  K = c_a c_b exp(-za zb/p |AB|^2).
struct PrimPairs {
    const double *p, *Px, *Py, *Pz, *K, *za;
    const float *fp, *fPx, *fPy, *fPz, *fK, *fza;  // fp32 mirrors
    const float *fPA, *fPB;                        // fp32 P - A and P - B, [3][n] (x, y, z planes)
    long long n;                                   // records (plane stride of fPA / fPB)
};

struct DensArgs {
    int npair, nbf;
    const double *A[TG_MAX_PAIRS], *B[TG_MAX_PAIRS];
    const double *S[TG_MAX_PAIRS], *T[TG_MAX_PAIRS];  // A + A^T, B + B^T
    double cJ[TG_MAX_PAIRS], cK[TG_MAX_PAIRS], cKlr[TG_MAX_PAIRS];
    int use_lr;
    double omega;
};

struct GeoArgs {
    int natom, nshell;
    const double *xyz;
    const int *sh_atom, *sh_bf;
};

struct ScreenArgs {
    double tau;         // 0: keep all
    double scale;       // 8 * npair
    const double *M;    // nshell x nshell block factors
    int nshell;
    int rank, nranks;
};

// Everything a class kernel needs about one molecule; kernels read it from
// a device array indexed by the tile's molecule id.
struct MolDesc {
    GeoArgs geo;
    DensArgs den;
    ScreenArgs scr;
    PrimPairs pp;
    PairSet sets[NPC];
    int atom_off;  // first atom of this molecule in the batch gradient
    int pad;
};

struct ClassLaunch {
    int P, Q;                  // bra and ket pair classes (same list iff P == Q)
    long long ntiles;
    const uint4 *tiles;        // (molecule, bra tile, ket tile, 0), grouped by molecule; tile t at tiles[t * stride]
    long long stride;          // 1, or nranks for tile-cyclic shards
    int nsplit;                // units per tile along the bra primitive pairs (>= 1)
    int nchunk;                // cooperative kernel: quartet chunks per tile (divides TILE / groups)
    int kind;                  // 0: default form of the class, 1: thread, 2: group, 3: warp
    int split_req;             // bra-primitive splits per tile requested by the autotuner (0: automatic)
};

struct OutArgs {
    double *partials;                 // [gridDim][natom_total*3], accumulated
    int natom_total;                  // atoms of the whole batch
    int natom_max;                    // atoms of the largest molecule
    unsigned long long *counters;     // NCNT per class (see NCNT)
    int use_smem;                     // per-molecule partial gradient kept in shared memory
    double *dump;                     // nullable: per-quartet gradients [tile][TILE][12] instead of reducing
    double *fock;                     // Fock build: the nbf x nbf output (atomic adds)
};

// Deterministic reduction of one staged tile into the per-molecule partial
// gradient tgt[atom*3 + i].  stg[q*12 + X*3 + i] holds quartet q's gradient
// on centre X (A, B, C, D); sat[q*4 + X] its atom (-1: quartet not computed).
// Quartet q = b*TK + j has bra pair row b and ket pair column j, so the A/B
// parts of a row and the C/D parts of a column share their atoms: rows and
// columns are summed in parallel first, then three threads (one per
// component) add the 2*TB + 2*TK sums in a fixed order.  red: 6*(TB+TK)
// doubles and 2*(TB+TK) ints of scratch.  All TILE threads must call it.
__device__ __forceinline__ void tile_reduce(const double *stg, const int *sat, double *red, int *ratom, double *tgt)
{
    const int t = threadIdx.x;
    for (int w = t; w < 6 * (TB + TK); w += TILE) {
        if (w < TB * 6) {  // row b, centre X in {A, B}, component i
            const int b = w / 6, X = (w % 6) / 3, i = w % 3;
            double s = 0.0;
            int a = -1;
            for (int j = 0; j < TK; ++j) {
                const int q = b * TK + j;
                s += stg[q * 12 + X * 3 + i];
                if (a < 0) a = sat[q * 4 + X];
            }
            red[w] = s;
            if (i == 0) ratom[b * 2 + X] = a;
        } else {  // column j, centre X in {C, D}, component i
            const int u = w - TB * 6, j = u / 6, X = 2 + (u % 6) / 3, i = u % 3;
            double s = 0.0;
            int a = -1;
            for (int b = 0; b < TB; ++b) {
                const int q = b * TK + j;
                s += stg[q * 12 + X * 3 + i];
                if (a < 0) a = sat[q * 4 + X];
            }
            red[w] = s;
            if (i == 0) ratom[TB * 2 + j * 2 + (X - 2)] = a;
        }
    }
    __syncthreads();
    if (t < 3) {
        for (int r = 0; r < 2 * (TB + TK); ++r) {
            const int a = ratom[r];
            if (a >= 0) tgt[a * 3 + t] += red[r * 3 + t];
        }
    }
}

// ---------------------------------------------------------------- Boys
// F_m(T) for m = 0..M (M <= BOYS_M - BOYS_TAYLOR).  T < 36: Taylor expansion
// of the top order about the nearest grid point, F_m(T0-d) = sum_k F_{m+k}(T0) d^k/k!,
// then downward recursion F_{m} = (2T F_{m+1} + e^-T)/(2m+1).  T >= 36: F_0 =
// sqrt(pi/T)/2 (erfc(6) < 3e-17) and upward recursion.
template <int M>
__device__ __forceinline__ void boys_fp64(double T, double (&F)[M + 1], const double *__restrict__ tab)
{
    if (T < BOYS_TMAX) {
        int i = __double2int_rn(T * (1.0 / BOYS_H));
        double d = i * BOYS_H - T;
        const double *row = tab + i * (BOYS_M + 1) + M;
        double acc = row[BOYS_TAYLOR];
#pragma unroll
        for (int k = BOYS_TAYLOR - 1; k >= 0; --k) acc = row[k] + acc * d * (1.0 / (k + 1));
        F[M] = acc;
        double et = exp(-T);
        double t2 = 2.0 * T;
#pragma unroll
        for (int m = M - 1; m >= 0; --m) F[m] = (t2 * F[m + 1] + et) * (1.0 / (2 * m + 1));
    } else {
        double it = 1.0 / T;
        F[0] = 0.88622692545275801365 * sqrt(it);
        double et = exp(-T);
        double h = 0.5 * it;
#pragma unroll
        for (int m = 0; m < M; ++m) F[m + 1] = ((2 * m + 1) * F[m] - et) * h;
    }
}

// ------------------------------------------------------- Hermite R tensor
// R^{(0)}_{tuv} for t+u+v <= LM (McMurchie-Davidson), in place from the
// bases R^{(n)}_{000} = base[n]:
//   R^{(n)}_{t,u,v} = (t-1) R^{(n+1)}_{t-2,u,v} + X R^{(n+1)}_{t-1,u,v}   (t > 0)
// and likewise along y, z.  Totals are updated high to low within a level, so
// every read still sees level n+1.
template <int LM, typename F>
__device__ __forceinline__ void hermite_R(F (&R)[nherm(LM)], const F (&base)[LM + 1], F X, F Y, F Z)
{
    R[0] = base[LM];
#pragma unroll
    for (int n = LM - 1; n >= 0; --n) {
#pragma unroll
        for (int k = LM - n; k >= 1; --k) {
#pragma unroll
            for (int t = 0; t <= k; ++t) {
#pragma unroll
                for (int u = 0; u <= k - t; ++u) {
                    const int v = k - t - u;
                    F r;
                    if (t > 0) {
                        r = X * R[hidx(t - 1, u, v)];
                        if (t > 1) r += F(t - 1) * R[hidx(t - 2, u, v)];
                    } else if (u > 0) {
                        r = Y * R[hidx(t, u - 1, v)];
                        if (u > 1) r += F(u - 1) * R[hidx(t, u - 2, v)];
                    } else {
                        r = Z * R[hidx(t, u, v - 1)];
                        if (v > 1) r += F(v - 1) * R[hidx(t, u, v - 2)];
                    }
                    R[hidx(t, u, v)] = r;
                }
            }
        }
        R[0] = base[n];
    }
}

// 1-D Hermite expansion coefficients E^{ij}_t (i <= I, j <= J) of a Gaussian
// product, without the exp(-ab/p AB^2) factor:
//   E^{i+1,j}_t = E^{ij}_{t-1}/(2p) + X_PA E^{ij}_t + (t+1) E^{ij}_{t+1}, same with X_PB for j.
template <int I, int J, typename F>
__device__ __forceinline__ void etab(F (&E)[I + 1][J + 1][I + J + 1], F PA, F PB, F oo2p)
{
#pragma unroll
    for (int i = 0; i <= I; ++i)
#pragma unroll
        for (int j = 0; j <= J; ++j)
#pragma unroll
            for (int t = 0; t <= I + J; ++t) E[i][j][t] = F(0);
    E[0][0][0] = F(1);
#pragma unroll
    for (int i = 0; i < I; ++i)
#pragma unroll
        for (int t = 0; t <= i + 1; ++t) {
            F v = F(0);
            if (t <= i) v = PA * E[i][0][t];
            if (t >= 1) v += oo2p * E[i][0][t - 1];
            if (t + 1 <= i) v += F(t + 1) * E[i][0][t + 1];
            E[i + 1][0][t] = v;
        }
#pragma unroll
    for (int j = 0; j < J; ++j)
#pragma unroll
        for (int i = 0; i <= I; ++i)
#pragma unroll
            for (int t = 0; t <= i + j + 1; ++t) {
                F v = F(0);
                if (t <= i + j) v = PB * E[i][j][t];
                if (t >= 1) v += oo2p * E[i][j][t - 1];
                if (t + 1 <= i + j) v += F(t + 1) * E[i][j][t + 1];
                E[i][j + 1][t] = v;
            }
}


// Algorithmic FLOPs of class qc per primitive quartet and per bra primitive
// pair visit (flops.cu; see tg_class_flops in tdgrad.h).
void class_flops(int qc, int nops, double *per_pq, double *per_p);

}  // namespace tg
