// Learned block router: tile features, MLP inference, and the training loop
// (forward + backward, fixed-order gradient reduction, Adam), all on the GPU.
// The router predicts log10 of a quartet tile's largest gradient
// contribution; it only decides fp32 vs fp64 for a tile and never skips work.
#include "router.cuh"

namespace tg {

__device__ __forceinline__ float lg10(double x) { return (float)log10(x > 1e-300 ? x : 1e-300); }

// 16 features of one quartet tile (TB bra pairs x TK ket pairs of one class).
__global__ void k_tile_features(int ntiles, const TileRef *tiles, FeatureArgs fa, float *feat)
{
    const int it = blockIdx.x * blockDim.x + threadIdx.x;
    if (it >= ntiles) return;
    const TileRef t = tiles[it];
    const PairSet &bra = fa.sets[t.P], &ket = fa.sets[t.Q];
    const int b0 = t.bt * TB, b1 = min(bra.n, b0 + TB), k0 = t.kt * TK, k1 = min(ket.n, k0 + TK);
    double qb = 0, qdb = 0, qk = 0, qdk = 0, mb = 0, mk = 0, mx = 0, ab = 0, cd = 0, pb = 1e300, pk = 1e300;
    double dmin = 1e300;
    const int ns = fa.nshell;
    for (int i = b0; i < b1; ++i) {
        qb = fmax(qb, bra.Q[i]);
        qdb = fmax(qdb, bra.Qd[i]);
        const int a = bra.sa[i], b = bra.sb[i];
        mb = fmax(mb, fa.M[(size_t)a * ns + b]);
        const double *A = fa.xyz + 3 * fa.sh_atom[a], *B = fa.xyz + 3 * fa.sh_atom[b];
        const double r = sqrt((A[0] - B[0]) * (A[0] - B[0]) + (A[1] - B[1]) * (A[1] - B[1]) + (A[2] - B[2]) * (A[2] - B[2]));
        ab = fmax(ab, r);
        for (int k = 0; k < bra.np[i]; ++k) pb = fmin(pb, fa.pp_p[bra.poff[i] + k]);
    }
    for (int j = k0; j < k1; ++j) {
        qk = fmax(qk, ket.Q[j]);
        qdk = fmax(qdk, ket.Qd[j]);
        const int c = ket.sa[j], d = ket.sb[j];
        mk = fmax(mk, fa.M[(size_t)c * ns + d]);
        const double *C = fa.xyz + 3 * fa.sh_atom[c], *D = fa.xyz + 3 * fa.sh_atom[d];
        const double r = sqrt((C[0] - D[0]) * (C[0] - D[0]) + (C[1] - D[1]) * (C[1] - D[1]) + (C[2] - D[2]) * (C[2] - D[2]));
        cd = fmax(cd, r);
        for (int k = 0; k < ket.np[j]; ++k) pk = fmin(pk, fa.pp_p[ket.poff[j] + k]);
    }
    for (int i = b0; i < b1; ++i) {
        const int a = bra.sa[i], b = bra.sb[i];
        const double *A = fa.xyz + 3 * fa.sh_atom[a], *B = fa.xyz + 3 * fa.sh_atom[b];
        for (int j = k0; j < k1; ++j) {
            const int c = ket.sa[j], d = ket.sb[j];
            mx = fmax(mx, fa.M[(size_t)a * ns + c]);
            mx = fmax(mx, fa.M[(size_t)a * ns + d]);
            mx = fmax(mx, fa.M[(size_t)b * ns + c]);
            mx = fmax(mx, fa.M[(size_t)b * ns + d]);
            const double *C = fa.xyz + 3 * fa.sh_atom[c], *D = fa.xyz + 3 * fa.sh_atom[d];
            double dd = 0.0;
            for (int x = 0; x < 3; ++x) {
                const double u = 0.5 * (A[x] + B[x]) - 0.5 * (C[x] + D[x]);
                dd += u * u;
            }
            dmin = fmin(dmin, dd);
        }
    }
    const double Mt = fmax(fmax(mb, mk), mx);
    const double bnd = fa.scale * fmax(qdb * qk, qb * qdk) * Mt * Mt;
    float *f = feat + (size_t)it * NFEAT;
    f[0] = (float)(pc_la(t.P) + pc_lb(t.P) + pc_la(t.Q) + pc_lb(t.Q)) * 0.125f;
    f[1] = lg10(bnd);
    f[2] = lg10(qb);
    f[3] = lg10(qk);
    f[4] = lg10(qdb);
    f[5] = lg10(qdk);
    f[6] = lg10(mx);
    f[7] = lg10(mb);
    f[8] = lg10(mk);
    f[9] = (float)(sqrt(dmin) * 0.1);
    f[10] = (float)(ab * 0.1);
    f[11] = (float)(cd * 0.1);
    f[12] = lg10(pb);
    f[13] = lg10(pk);
    f[14] = log2f((float)bra.np[b0]);
    f[15] = log2f((float)ket.np[k0]);
}

// Feature standardisation statistics (mean, std) in a fixed order.
__global__ void k_feature_stats(int n, const float *X, float *mu, float *sd)
{
    const int j = threadIdx.x;
    if (j >= NFEAT) return;
    double s = 0.0, s2 = 0.0;
    for (int i = 0; i < n; ++i) {
        const double v = X[(size_t)i * NFEAT + j];
        s += v;
        s2 += v * v;
    }
    const double m = n > 0 ? s / n : 0.0;
    const double var = n > 0 ? s2 / n - m * m : 1.0;
    mu[j] = (float)m;
    sd[j] = (float)sqrt(var > 1e-12 ? var : 1.0);
}

__device__ __forceinline__ void mlp_forward(const float *w, const float *x, float *h1, float *h2, float &y)
{
    const float *W1 = w, *b1 = W1 + NH * NFEAT, *W2 = b1 + NH, *b2 = W2 + NH * NH, *w3 = b2 + NH, *b3 = w3 + NH;
    for (int i = 0; i < NH; ++i) {
        float a = b1[i];
        for (int j = 0; j < NFEAT; ++j) a += W1[i * NFEAT + j] * x[j];
        h1[i] = tanhf(a);
    }
    for (int i = 0; i < NH; ++i) {
        float a = b2[i];
        for (int j = 0; j < NH; ++j) a += W2[i * NH + j] * h1[j];
        h2[i] = tanhf(a);
    }
    float a = b3[0];
    for (int j = 0; j < NH; ++j) a += w3[j] * h2[j];
    y = a;
}

__global__ void k_mlp_predict(int n, const float *X, const float *mu, const float *sd, const float *params, float *out)
{
    __shared__ float w[NPARAM];
    for (int k = threadIdx.x; k < NPARAM; k += blockDim.x) w[k] = params[k];
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float x[NFEAT], h1[NH], h2[NH], y;
    for (int j = 0; j < NFEAT; ++j) x[j] = (X[(size_t)i * NFEAT + j] - mu[j]) / sd[j];
    mlp_forward(w, x, h1, h2, y);
    out[i] = y;
}

// Forward + backward of the expectile loss for TRB samples per block; the
// block's parameter gradient (sum over its samples, divided by n) and loss
// go to partial slots, reduced later in a fixed order.
__global__ void __launch_bounds__(TRB) k_mlp_fwd_bwd(int n, const float *X, const float *y, const float *mu,
                                                     const float *sd, const float *params, float q, float *gpart,
                                                     float *lpart)
{
    extern __shared__ float sm[];
    float *w = sm;                          // NPARAM
    float *sx = w + NPARAM;                 // TRB x NFEAT
    float *s1 = sx + TRB * NFEAT;           // TRB x NH  (h1, then da1)
    float *s2 = s1 + TRB * NH;              // TRB x NH  (h2, then da2)
    float *sdy = s2 + TRB * NH;             // TRB
    float *sl = sdy + TRB;                  // TRB
    float *sa1 = sl + TRB;                  // TRB x NH (da1)
    for (int k = threadIdx.x; k < NPARAM; k += blockDim.x) w[k] = params[k];
    __syncthreads();
    const int s = threadIdx.x;
    const int i = blockIdx.x * TRB + s;
    const float *W2 = w + NH * NFEAT + NH, *w3 = W2 + NH * NH + NH;
    if (i < n) {
        float x[NFEAT], h1[NH], h2[NH], yh;
        for (int j = 0; j < NFEAT; ++j) x[j] = (X[(size_t)i * NFEAT + j] - mu[j]) / sd[j];
        mlp_forward(w, x, h1, h2, yh);
        const float r = y[i] - yh;
        const float wt = r > 0.f ? q : 1.f - q;
        sl[s] = wt * r * r / n;
        const float dy = -2.f * wt * r / n;
        sdy[s] = dy;
        float da2[NH];
        for (int k = 0; k < NH; ++k) da2[k] = dy * w3[k] * (1.f - h2[k] * h2[k]);
        for (int j = 0; j < NH; ++j) {
            float a = 0.f;
            for (int k = 0; k < NH; ++k) a += W2[k * NH + j] * da2[k];
            sa1[s * NH + j] = a * (1.f - h1[j] * h1[j]);
        }
        for (int j = 0; j < NFEAT; ++j) sx[s * NFEAT + j] = x[j];
        for (int k = 0; k < NH; ++k) {
            s1[s * NH + k] = h1[k];
            s2[s * NH + k] = h2[k];
        }
        for (int k = 0; k < NH; ++k) s2[s * NH + k] = h2[k];
        // da2 kept in a second pass below through s2 (h2) and sdy
    } else {
        sl[s] = 0.f;
        sdy[s] = 0.f;
        for (int j = 0; j < NFEAT; ++j) sx[s * NFEAT + j] = 0.f;
        for (int k = 0; k < NH; ++k) {
            s1[s * NH + k] = 0.f;
            s2[s * NH + k] = 0.f;
            sa1[s * NH + k] = 0.f;
        }
    }
    __syncthreads();
    const int nvalid = min(TRB, n - blockIdx.x * TRB);
    float *gp = gpart + (size_t)blockIdx.x * NPARAM;
    // each thread owns parameters k = threadIdx.x + m*TRB and sums over the block's samples in order
    for (int k = threadIdx.x; k < NPARAM; k += TRB) {
        float acc = 0.f;
        if (k < NH * NFEAT) {  // W1[i][j] += da1[i] x[j]
            const int ii = k / NFEAT, j = k % NFEAT;
            for (int t = 0; t < nvalid; ++t) acc += sa1[t * NH + ii] * sx[t * NFEAT + j];
        } else if (k < NH * NFEAT + NH) {  // b1
            const int ii = k - NH * NFEAT;
            for (int t = 0; t < nvalid; ++t) acc += sa1[t * NH + ii];
        } else if (k < NH * NFEAT + NH + NH * NH) {  // W2[i][j] += da2[i] h1[j]
            const int kk = k - NH * NFEAT - NH, ii = kk / NH, j = kk % NH;
            for (int t = 0; t < nvalid; ++t) {
                const float h2v = s2[t * NH + ii];
                const float da2 = sdy[t] * w3[ii] * (1.f - h2v * h2v);
                acc += da2 * s1[t * NH + j];
            }
        } else if (k < NH * NFEAT + NH + NH * NH + NH) {  // b2
            const int ii = k - NH * NFEAT - NH - NH * NH;
            for (int t = 0; t < nvalid; ++t) {
                const float h2v = s2[t * NH + ii];
                acc += sdy[t] * w3[ii] * (1.f - h2v * h2v);
            }
        } else if (k < NPARAM - 1) {  // w3
            const int ii = k - NH * NFEAT - NH - NH * NH - NH;
            for (int t = 0; t < nvalid; ++t) acc += sdy[t] * s2[t * NH + ii];
        } else {  // b3
            for (int t = 0; t < nvalid; ++t) acc += sdy[t];
        }
        gp[k] = acc;
    }
    if (threadIdx.x == 0) {
        float L = 0.f;
        for (int t = 0; t < nvalid; ++t) L += sl[t];
        lpart[blockIdx.x] = L;
    }
}

__global__ void k_sum_partials(int nblocks, int width, const float *part, float *out)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= width) return;
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += part[(size_t)b * width + k];
    out[k] = (float)s;
}

__global__ void k_adam(int n, float *params, const float *grad, float *m, float *v, float lr, float b1, float b2,
                       float eps, int step)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const float g = grad[k];
    const float mk = b1 * m[k] + (1.f - b1) * g;
    const float vk = b2 * v[k] + (1.f - b2) * g * g;
    m[k] = mk;
    v[k] = vk;
    const float mh = mk / (1.f - powf(b1, (float)step));
    const float vh = vk / (1.f - powf(b2, (float)step));
    params[k] -= lr * mh / (sqrtf(vh) + eps);
}

}  // namespace tg
