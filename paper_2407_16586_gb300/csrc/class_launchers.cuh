// Launchers of the 21 class kernels, one translation unit each.
#pragma once
#include "tg_internal.cuh"

namespace tg {

typedef cudaError_t (*class_launcher)(int fp32, int grid, size_t smem, cudaStream_t st, const MolDesc *mols,
                                      const ClassLaunch &cl, const OutArgs &out, const double *boys);

cudaError_t launch_qc00(int, int, size_t, cudaStream_t, const MolDesc *, const ClassLaunch &, const OutArgs &,
                         const double *);
cudaError_t launch_qc01(int, int, size_t, cudaStream_t, const MolDesc *, const ClassLaunch &, const OutArgs &,
                         const double *);
cudaError_t launch_qc02(int, int, size_t, cudaStream_t, const MolDesc *, const ClassLaunch &, const OutArgs &,
                         const double *);
cudaError_t launch_qc03(int, int, size_t, cudaStream_t, const MolDesc *, const ClassLaunch &, const OutArgs &,
                         const double *);
cudaError_t launch_qc04(int, int, size_t, cudaStream_t, const MolDesc *, const ClassLaunch &, const OutArgs &,
                         const double *);
cudaError_t launch_qc05(int, int, size_t, cudaStream_t, const MolDesc *, const ClassLaunch &, const OutArgs &,
                         const double *);
cudaError_t launch_qc06(int, int, size_t, cudaStream_t, const MolDesc *, const ClassLaunch &, const OutArgs &,
                         const double *);
cudaError_t launch_qc07(int, int, size_t, cudaStream_t, const MolDesc *, const ClassLaunch &, const OutArgs &,
                         const double *);
cudaError_t launch_qc08(int, int, size_t, cudaStream_t, const MolDesc *, const ClassLaunch &, const OutArgs &,
                         const double *);
cudaError_t launch_qc09(int, int, size_t, cudaStream_t, const MolDesc *, const ClassLaunch &, const OutArgs &,
                         const double *);
cudaError_t launch_qc10(int, int, size_t, cudaStream_t, const MolDesc *, const ClassLaunch &, const OutArgs &,
                         const double *);
cudaError_t launch_qc11(int, int, size_t, cudaStream_t, const MolDesc *, const ClassLaunch &, const OutArgs &,
                         const double *);
cudaError_t launch_qc12(int, int, size_t, cudaStream_t, const MolDesc *, const ClassLaunch &, const OutArgs &,
                         const double *);
cudaError_t launch_qc13(int, int, size_t, cudaStream_t, const MolDesc *, const ClassLaunch &, const OutArgs &,
                         const double *);
cudaError_t launch_qc14(int, int, size_t, cudaStream_t, const MolDesc *, const ClassLaunch &, const OutArgs &,
                         const double *);
cudaError_t launch_qc15(int, int, size_t, cudaStream_t, const MolDesc *, const ClassLaunch &, const OutArgs &,
                         const double *);
cudaError_t launch_qc16(int, int, size_t, cudaStream_t, const MolDesc *, const ClassLaunch &, const OutArgs &,
                         const double *);
cudaError_t launch_qc17(int, int, size_t, cudaStream_t, const MolDesc *, const ClassLaunch &, const OutArgs &,
                         const double *);
cudaError_t launch_qc18(int, int, size_t, cudaStream_t, const MolDesc *, const ClassLaunch &, const OutArgs &,
                         const double *);
cudaError_t launch_qc19(int, int, size_t, cudaStream_t, const MolDesc *, const ClassLaunch &, const OutArgs &,
                         const double *);
cudaError_t launch_qc20(int, int, size_t, cudaStream_t, const MolDesc *, const ClassLaunch &, const OutArgs &,
                         const double *);

// Fock-type build (fp64): one launcher per class
typedef cudaError_t (*fock_launcher)(int grid, cudaStream_t st, const MolDesc *mols, const ClassLaunch &cl,
                                     const OutArgs &out, const double *boys);
cudaError_t launch_fock_qc00(int, cudaStream_t, const MolDesc *, const ClassLaunch &, const OutArgs &,
                              const double *);
cudaError_t launch_fock_qc01(int, cudaStream_t, const MolDesc *, const ClassLaunch &, const OutArgs &,
                              const double *);
cudaError_t launch_fock_qc02(int, cudaStream_t, const MolDesc *, const ClassLaunch &, const OutArgs &,
                              const double *);
cudaError_t launch_fock_qc03(int, cudaStream_t, const MolDesc *, const ClassLaunch &, const OutArgs &,
                              const double *);
cudaError_t launch_fock_qc04(int, cudaStream_t, const MolDesc *, const ClassLaunch &, const OutArgs &,
                              const double *);
cudaError_t launch_fock_qc05(int, cudaStream_t, const MolDesc *, const ClassLaunch &, const OutArgs &,
                              const double *);
cudaError_t launch_fock_qc06(int, cudaStream_t, const MolDesc *, const ClassLaunch &, const OutArgs &,
                              const double *);
cudaError_t launch_fock_qc07(int, cudaStream_t, const MolDesc *, const ClassLaunch &, const OutArgs &,
                              const double *);
cudaError_t launch_fock_qc08(int, cudaStream_t, const MolDesc *, const ClassLaunch &, const OutArgs &,
                              const double *);
cudaError_t launch_fock_qc09(int, cudaStream_t, const MolDesc *, const ClassLaunch &, const OutArgs &,
                              const double *);
cudaError_t launch_fock_qc10(int, cudaStream_t, const MolDesc *, const ClassLaunch &, const OutArgs &,
                              const double *);
cudaError_t launch_fock_qc11(int, cudaStream_t, const MolDesc *, const ClassLaunch &, const OutArgs &,
                              const double *);
cudaError_t launch_fock_qc12(int, cudaStream_t, const MolDesc *, const ClassLaunch &, const OutArgs &,
                              const double *);
cudaError_t launch_fock_qc13(int, cudaStream_t, const MolDesc *, const ClassLaunch &, const OutArgs &,
                              const double *);
cudaError_t launch_fock_qc14(int, cudaStream_t, const MolDesc *, const ClassLaunch &, const OutArgs &,
                              const double *);
cudaError_t launch_fock_qc15(int, cudaStream_t, const MolDesc *, const ClassLaunch &, const OutArgs &,
                              const double *);
cudaError_t launch_fock_qc16(int, cudaStream_t, const MolDesc *, const ClassLaunch &, const OutArgs &,
                              const double *);
cudaError_t launch_fock_qc17(int, cudaStream_t, const MolDesc *, const ClassLaunch &, const OutArgs &,
                              const double *);
cudaError_t launch_fock_qc18(int, cudaStream_t, const MolDesc *, const ClassLaunch &, const OutArgs &,
                              const double *);
cudaError_t launch_fock_qc19(int, cudaStream_t, const MolDesc *, const ClassLaunch &, const OutArgs &,
                              const double *);
cudaError_t launch_fock_qc20(int, cudaStream_t, const MolDesc *, const ClassLaunch &, const OutArgs &,
                              const double *);
static const fock_launcher kFockLaunchers[NQC] = {
    launch_fock_qc00, launch_fock_qc01, launch_fock_qc02, launch_fock_qc03, launch_fock_qc04, launch_fock_qc05, launch_fock_qc06, launch_fock_qc07, launch_fock_qc08, launch_fock_qc09, launch_fock_qc10, launch_fock_qc11, launch_fock_qc12, launch_fock_qc13, launch_fock_qc14, launch_fock_qc15, launch_fock_qc16, launch_fock_qc17, launch_fock_qc18, launch_fock_qc19, launch_fock_qc20};

static const class_launcher kClassLaunchers[NQC] = {
    launch_qc00, launch_qc01, launch_qc02, launch_qc03, launch_qc04, launch_qc05, launch_qc06, launch_qc07, launch_qc08, launch_qc09, launch_qc10, launch_qc11, launch_qc12, launch_qc13, launch_qc14, launch_qc15, launch_qc16, launch_qc17, launch_qc18, launch_qc19, launch_qc20};

}  // namespace tg
