// Algorithmic FLOP count of the class kernels' evaluation (host only).
//
// The count is that of the McMurchie-Davidson evaluation in the form the
// class kernels use (eri_warp.cuh): per primitive quartet, the Boys orders
// (six Taylor terms each), the Hermite R recursion of both operators, the
// ket products E^{cd} over their index boxes, W += E^{cd} R over the boxes of
// cd, z = F R over the derivative boxes of cd and the d/dC products; per bra
// primitive pair of a quartet, the bra products E^{ab}, F = Gamma E^{ab},
// Y = Gamma W over the derivative boxes of ab and the d/dA, d/dA + d/dB
// products.  An FMA counts 2, a multiply or add 1.  Index boxes: the
// expansion coefficient E^{ab}_{tuv} of a function pair vanishes unless
// t <= a_x + b_x, u <= a_y + b_y, v <= a_z + b_z (eq. cartG); the derivative
// of eq. deriv raises one of the three limits by one.
#include "tg_internal.cuh"

namespace tg {
namespace {

int box_count(const int n[3]) { return (n[0] + 1) * (n[1] + 1) * (n[2] + 1); }

// number of the three derivative boxes of extent n that contain (t, u, v)
int deriv_boxes(const int n[3], int t, int u, int v)
{
    const bool inx = t <= n[0], iny = u <= n[1], inz = v <= n[2];
    return (int)(t <= n[0] + 1 && iny && inz) + (int)(inx && u <= n[1] + 1 && inz) +
           (int)(inx && iny && v <= n[2] + 1);
}

// summed extents of the function pairs of shells la, lb
template <typename Fn>
void for_pair_extents(int la, int lb, Fn &&fn)
{
    for (int ca = 0; ca < ncart(la); ++ca)
        for (int cb = 0; cb < ncart(lb); ++cb) {
            int a[3], b[3];
            const int sa = ca == 0 ? 0 : (ca < 3 ? 1 : 2), sb = cb == 0 ? 0 : (cb < 3 ? 1 : 2);
            a[2] = ca - sa * (sa + 1) / 2;
            a[1] = sa - a[2];
            a[0] = la - sa;
            b[2] = cb - sb * (sb + 1) / 2;
            b[1] = sb - b[2];
            b[0] = lb - sb;
            const int n[3] = {a[0] + b[0], a[1] + b[1], a[2] + b[2]};
            fn(n);
        }
}

}  // namespace

void class_flops(int qc, int nops, double *per_pq, double *per_p)
{
    int P = 0;
    while ((P + 1) * (P + 2) / 2 <= qc) ++P;
    const int Q = qc - P * (P + 1) / 2;
    const int la = pc_la(P), lb = pc_lb(P), lc = pc_la(Q), ld = pc_lb(Q);
    const int L1 = la + lb, L2 = lc + ld, L = L1 + L2;
    const int nab = ncart(la) * ncart(lb), ncd = ncart(lc) * ncart(ld);
    // R recursion: level n holds the totals 1 .. L+1-n; one multiply, plus an
    // FMA where the recursion has its second term
    double r = 0.0;
    for (int n = 0; n <= L; ++n)
        for (int k = 1; k <= L + 1 - n; ++k)
            for (int t = 0; t <= k; ++t)
                for (int u = 0; u <= k - t; ++u) {
                    const int v = k - t - u;
                    const bool two = t > 0 ? t > 1 : (u > 0 ? u > 1 : v > 1);
                    r += two ? 3.0 : 1.0;
                }
    double pq = nops * r + nops * (L + 2) * (6 * 2 + 2);
    double box_cd = 0.0, v_cd = 0.0, dc = 0.0;
    for_pair_extents(lc, ld, [&](const int n[3]) {
        box_cd += box_count(n);
        for (int t = 0; t <= n[0] + 1; ++t)
            for (int u = 0; u <= n[1] + 1; ++u)
                for (int v = 0; v <= n[2] + 1; ++v) {
                    const int g = deriv_boxes(n, t, u, v);
                    if (g) {
                        v_cd += 1.0;
                        dc += 7.0 * g;
                    }
                }
    });
    pq += 2.0 * box_cd + nops * box_cd * nherm(L1 + 1) * 2.0 + nops * v_cd * nherm(L1) * 2.0 + dc;
    double box_ab = 0.0, v_ab = 0.0, da = 0.0;
    for_pair_extents(la, lb, [&](const int n[3]) {
        box_ab += box_count(n);
        for (int t = 0; t <= n[0] + 1; ++t)
            for (int u = 0; u <= n[1] + 1; ++u)
                for (int v = 0; v <= n[2] + 1; ++v) {
                    const int g = deriv_boxes(n, t, u, v);
                    if (g) {
                        v_ab += 1.0;
                        da += 11.0 * g;
                    }
                }
    });
    const double p = 2.0 * box_ab + nops * ncd * box_ab * 2.0 + nops * ncd * v_ab * 2.0 + da;
    (void)nab;
    *per_pq = pq;
    *per_p = p;
}

}  // namespace tg

extern "C" int tg_class_flops(int qc, int nops, double *per_prim_quartet, double *per_bra_prim)
{
    if (qc < 0 || qc >= tg::NQC || (nops != 1 && nops != 2) || !per_prim_quartet || !per_bra_prim) return TG_EINVAL;
    tg::class_flops(qc, nops, per_prim_quartet, per_bra_prim);
    return TG_OK;
}
