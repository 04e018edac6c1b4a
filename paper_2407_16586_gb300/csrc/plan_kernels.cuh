// Device block screen, tile lists and routing of one call (plan_kernels.cu).
#pragma once
#include <cmath>

#include "router.cuh"

namespace tg {

constexpr int GROUP = 32;  // ket tiles per group of the hierarchical screen

// Maxima of Q, Q' and the density factor over the tiles of one pair class
// (bra tiles of TB pairs: bq, bqd, bm; ket tiles of TK pairs: kq, kqd, km;
// groups of GROUP ket tiles: gq, gqd, gm).
struct TileMaxima {
    const double *bq, *bqd, *bm;
    const double *kq, *kqd, *km;
    const double *gq, *gqd, *gm;
    int nbt, nkt;
};

struct RowArgs {
    int nrows;
    const int4 *rows;  // (class, bra tile, first ket tile, end ket tile): ket tiles of equal cost
    TileMaxima t[NPC];
    int qcP[NQC], qcQ[NQC];
    double tau, scale;
    int fock;  // 1: Fock-build bound scale * Q_bt Q_kt * max(M_bt, M_kt)
};

// Routing bins: 8 per octave of the fp32 error estimate e; bin 0 holds e <= 2^-1000.
constexpr int RBIN_PER_OCTAVE = 8;
constexpr int RBIN_OFFSET = 8001;
constexpr int RBIN_N = 8704;
__host__ __device__ inline int route_bin(double e)
{
    if (!(e > 0x1p-1000)) return 0;
    int b = (int)floor(log2(e) * RBIN_PER_OCTAVE) + RBIN_OFFSET;
    return b < 1 ? 1 : (b > RBIN_N - 1 ? RBIN_N - 1 : b);
}
// upper edge of bin b (e < upper for every e in the bin)
inline double route_bin_upper(int b) { return b == 0 ? 0x1p-1000 : std::exp2((double)(b - RBIN_OFFSET + 1) / RBIN_PER_OCTAVE); }

__global__ void k_tile_maxima(int n, int bsz, const int *sa, const int *sb, const double *Q, const double *Qd,
                              const double *Mrow, double *tq, double *tqd, double *tm);
__global__ void k_group_maxima(int nt, const double *tq, const double *tqd, const double *tm, double *gq, double *gqd,
                               double *gm);
__global__ void k_tile_rows(RowArgs a, int mode, int *count, const long long *off, uint4 *tiles, float *bnd);
__global__ void k_tile_refs(long long n, const uint4 *tiles, RowArgs a, TileRef *refs);
__global__ void k_route_bins(long long n, const uint4 *tiles, const float *val, int kind, double c0, double c1,
                             RowArgs a, int *bin, unsigned long long *hist);
__global__ void k_row_fp32_count(int nrows, const long long *off, const long long *base, int srank, int snr,
                                 const int *bin, int cut, int *cnt32, int *cntk);
__global__ void k_row_scatter(int nrows, const long long *off, const long long *base, int srank, int snr,
                              const uint4 *tiles, const int *bin, int cut, const long long *o64, const long long *o32,
                              uint4 *out);

}  // namespace tg
