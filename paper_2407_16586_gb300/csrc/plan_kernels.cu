// Device side of the block screen, the angular-class tile lists and the
// fp32 / fp64 routing of one call (Sec. II.C: pair lists presorted per
// angular class and cut into equal blocks; Sec. II.E: Schwarz x density
// screening of every block of quartets).
//
// A class's sorted pair list is cut into bra tiles of TB pairs and ket
// tiles of TK pairs.  The bound of a tile (bra tile bt, ket tile kt) is
//   scale * max(Q'_bt Q_kt, Q_bt Q'_kt) * max(M_bt, M_kt)^2,
// with Q, Q', M the maxima over the tile's pairs (M: the largest block
// density factor of a pair's shells); a tile is kept iff its bound is at
// least tau.  Ket tiles are grouped by GROUP: the bound of a group (maxima
// over its tiles) is no smaller than the bound of any of its tiles, so a
// group below tau is skipped whole (the hierarchical screen).  One thread
// walks one row -- a bra tile and a run of ket tiles of one cost (the
// primitive-pair counts of their first pairs) -- in increasing ket tile
// order, first counting, then writing at the row's offset; the rows come
// sorted by decreasing cost, so every class list is ordered by decreasing
// cost and is identical from run to run.
#include "plan_kernels.cuh"

namespace tg {

__global__ void k_tile_maxima(int n, int bsz, const int *__restrict__ sa, const int *__restrict__ sb,
                              const double *__restrict__ Q, const double *__restrict__ Qd,
                              const double *__restrict__ Mrow, double *tq, double *tqd, double *tm)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int nt = (n + bsz - 1) / bsz;
    if (t >= nt) return;
    double q = 0.0, qd = 0.0, m = 0.0;
    const int hi = min(n, (t + 1) * bsz);
    for (int i = t * bsz; i < hi; ++i) {
        q = fmax(q, Q[i]);
        qd = fmax(qd, Qd[i]);
        m = fmax(m, fmax(Mrow[sa[i]], Mrow[sb[i]]));
    }
    tq[t] = q;
    tqd[t] = qd;
    tm[t] = m;
}

__global__ void k_group_maxima(int nt, const double *__restrict__ tq, const double *__restrict__ tqd,
                               const double *__restrict__ tm, double *gq, double *gqd, double *gm)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g * GROUP >= nt) return;
    double q = 0.0, qd = 0.0, m = 0.0;
    const int hi = min(nt, (g + 1) * GROUP);
    for (int t = g * GROUP; t < hi; ++t) {
        q = fmax(q, tq[t]);
        qd = fmax(qd, tqd[t]);
        m = fmax(m, tm[t]);
    }
    gq[g] = q;
    gqd[g] = qd;
    gm[g] = m;
}

// mode 0: count[r] = kept tiles of row r; mode 1: write them at off[r]
__global__ void k_tile_rows(RowArgs a, int mode, int *count, const long long *off, uint4 *tiles, float *bnd)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= a.nrows) return;
    const int4 row = a.rows[r];
    const int qc = row.x, bt = row.y, k0 = row.z;
    const int P = a.qcP[qc], Q = a.qcQ[qc];
    const double q = a.t[P].bq[bt], qd = a.t[P].bqd[bt], m = a.t[P].bm[bt];
    const int nkt = row.w;  // end of the run (the host applies the canonical limit kt * TK <= bt * TB + TB - 1)
    const TileMaxima &K = a.t[Q];
    long long o = mode ? off[r] : 0;
    int c = 0;
    for (int g = k0 / GROUP; g * GROUP < nkt; ++g) {
        if (a.tau > 0.0) {
            const double Mt = fmax(m, K.gm[g]);
            const double b = a.fock ? a.scale * q * K.gq[g] * Mt : a.scale * fmax(qd * K.gq[g], q * K.gqd[g]) * Mt * Mt;
            if (b < a.tau) continue;
        }
        const int hi = min(nkt, (g + 1) * GROUP);
        for (int kt = max(k0, g * GROUP); kt < hi; ++kt) {
            const double Mt = fmax(m, K.km[kt]);
            const double b = a.fock ? a.scale * q * K.kq[kt] * Mt : a.scale * fmax(qd * K.kq[kt], q * K.kqd[kt]) * Mt * Mt;
            if (a.tau > 0.0 && b < a.tau) continue;
            if (mode) {
                tiles[o + c] = make_uint4(0u, (unsigned)bt, (unsigned)kt, (unsigned)qc);
                bnd[o + c] = (float)b;
            }
            ++c;
        }
    }
    if (!mode) count[r] = c;
}

__global__ void k_tile_refs(long long n, const uint4 *__restrict__ tiles, RowArgs a, TileRef *refs)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint4 t = tiles[i];
    TileRef r;
    r.P = a.qcP[t.w];
    r.Q = a.qcQ[t.w];
    r.bt = t.y;
    r.kt = t.z;
    refs[i] = r;
}

// Log-binned fp32 error estimate of every tile (see route_bin) and the
// count of tiles per bin.  kind 0: e = c0 * nfq(class) * bound; kind 1:
// e = c0 * 10^(prediction + c1).  Grid-stride with a per-block histogram in
// shared memory (32-bit counts, at most 2^31 tiles per launch), added to the
// global one bin by bin at the end, so the global atomics do not pile up on
// the few bins that hold most tiles.
__global__ void k_route_bins(long long n, const uint4 *__restrict__ tiles, const float *__restrict__ val, int kind,
                             double c0, double c1, RowArgs a, int *bin, unsigned long long *hist)
{
    extern __shared__ unsigned int sh_hist[];
    for (int k = threadIdx.x; k < RBIN_N; k += blockDim.x) sh_hist[k] = 0u;
    __syncthreads();
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        double e;
        if (kind == 0) {
            const int qc = tiles[i].w;
            const int P = a.qcP[qc], Q = a.qcQ[qc];
            const int nfq = ncart(pc_la(P)) * ncart(pc_lb(P)) * ncart(pc_la(Q)) * ncart(pc_lb(Q));
            e = c0 * nfq * (double)val[i];
        } else {
            e = c0 * pow(10.0, (double)val[i] + c1);
        }
        const int b = route_bin(e);
        bin[i] = b;
        atomicAdd(sh_hist + b, 1u);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < RBIN_N; k += blockDim.x)
        if (sh_hist[k]) atomicAdd(hist + k, (unsigned long long)sh_hist[k]);
}

// Tile shard (tg_options.shard_mode = TG_SHARD_TILES): tile i of the screened
// list belongs to rank (i - base of its class) mod snr, i.e. the class lists
// are dealt round-robin in their planner order BEFORE the fp32 / fp64 split,
// so a shard holds the same tiles at every precision and the route is the
// one of the whole list.
__device__ __forceinline__ bool in_shard(long long i, long long base, int srank, int snr)
{
    return snr <= 1 || (i - base) % snr == srank;
}

// Kept tiles of each row (cntk) and those of them routed to fp32 (cnt32): a
// tile goes to fp32 iff its bin is below the cut-off (bin == nullptr: every
// tile counts as bin 0, so cut 0 routes all to fp64 and any cut > 0 all to
// fp32).
__global__ void k_row_fp32_count(int nrows, const long long *__restrict__ off, const long long *__restrict__ base,
                                 int srank, int snr, const int *__restrict__ bin, int cut, int *cnt32, int *cntk)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrows) return;
    int c = 0, k = 0;
    for (long long i = off[r]; i < off[r + 1]; ++i) {
        if (!in_shard(i, base[r], srank, snr)) continue;
        ++k;
        c += ((bin ? bin[i] : 0) < cut) ? 1 : 0;
    }
    cnt32[r] = c;
    cntk[r] = k;
}

// Row r's kept tiles, in order, to its fp64 slots at o64[r] and its fp32
// slots at o32[r] of the launch list (molecule 0, bra tile, ket tile, 0).
__global__ void k_row_scatter(int nrows, const long long *__restrict__ off, const long long *__restrict__ base,
                              int srank, int snr, const uint4 *__restrict__ tiles, const int *__restrict__ bin, int cut,
                              const long long *__restrict__ o64, const long long *__restrict__ o32, uint4 *out)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrows) return;
    long long a = o64[r], b = o32[r];
    for (long long i = off[r]; i < off[r + 1]; ++i) {
        if (!in_shard(i, base[r], srank, snr)) continue;
        const uint4 t = tiles[i];
        const bool f32 = (bin ? bin[i] : 0) < cut;
        out[f32 ? b++ : a++] = make_uint4(0u, t.y, t.z, 0u);
    }
}

}  // namespace tg
