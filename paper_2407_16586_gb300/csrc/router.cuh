// Block router: features of quartet tiles and a 16-32-32-1 tanh MLP.
#pragma once
#include "tg_internal.cuh"

namespace tg {

constexpr int NFEAT = 16;
constexpr int NH = 32;
constexpr int NPARAM = NH * NFEAT + NH + NH * NH + NH + NH + 1;  // 1633
constexpr int TRB = 128;  // training samples per block

struct TileRef {
    int P, Q;        // bra and ket pair classes
    unsigned bt, kt; // tile indices in the class lists
};

struct FeatureArgs {
    PairSet sets[NPC];
    const double *M;      // nshell x nshell block density factors
    const double *xyz;
    const int *sh_atom;
    const double *pp_p;   // primitive-pair exponent sums
    int nshell;
    double scale;         // 8 * npair
};

__global__ void k_tile_features(int ntiles, const TileRef *tiles, FeatureArgs fa, float *feat);
__global__ void k_feature_stats(int n, const float *X, float *mu, float *sd);
__global__ void k_mlp_predict(int n, const float *X, const float *mu, const float *sd, const float *params, float *out);
__global__ void k_mlp_fwd_bwd(int n, const float *X, const float *y, const float *mu, const float *sd,
                              const float *params, float q, float *gpart, float *lpart);
__global__ void k_sum_partials(int nblocks, int width, const float *part, float *out);
__global__ void k_adam(int n, float *params, const float *grad, float *m, float *v, float lr, float b1, float b2,
                       float eps, int step);

constexpr size_t fwd_bwd_smem() { return sizeof(float) * (NPARAM + TRB * (NFEAT + 3 * NH + 2)); }

}  // namespace tg
