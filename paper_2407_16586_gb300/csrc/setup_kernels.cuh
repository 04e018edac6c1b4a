#pragma once
#include "tg_internal.cuh"

namespace tg {

__global__ void k_boys_table(double *tab);
__global__ void k_normalise(int nshell, const int *sh_l, const int *sh_nprim, const int *sh_poff,
                            const double *exps, const double *coefs, double *cn);
__global__ void k_schwarz(int npairs, const int2 *pairs, const double *xyz, const int *sh_atom, const int *sh_l,
                          const int *sh_nprim, const int *sh_poff, const double *exps, const double *cn, double *Q,
                          double *Qd, const long long *bpoff, double *bp);
__global__ void k_blockmax(int nshell, const int *sh_bf, const int *sh_l, DensArgs den, const double *w,
                           double *M, double *Mrow);
__global__ void k_rowmax(int nshell, const double *M, double *Mrow);
__global__ void k_prim_count(int npairs, const int *psa, const int *psb, const int *key, const int *sh_nprim,
                             const long long *bpoff, const double *bp, double scale, double qq, double mmax,
                             double eps_p, int *np_out);
__global__ void k_prim_pairs(int npairs, const int *psa, const int *psb, const int *poff, const int *key,
                             const double *xyz, const int *sh_atom, const int *sh_nprim, const int *sh_poff,
                             const double *exps, const double *cn, const long long *bpoff, const double *bp,
                             double scale, double qq, double mmax, double eps_p, double *p_, double *Px, double *Py,
                             double *Pz, double *K, double *za_, float *fp, float *fPx, float *fPy, float *fPz,
                             float *fK, float *fza, float *fPA, float *fPB, long long nrec);
__global__ void k_symm(int nbf, const double *A, double *S);
__global__ void k_fock_combine(int nbf, DensArgs den, double *SJ, double *BK, double *BL);
__global__ void k_reduce(int n, int nslab, const double *partials, double *grad);
__global__ void k_sph_to_cart(int nbf, int nsph, const int *cmap, const double *Asph, double *Acart);

}  // namespace tg
