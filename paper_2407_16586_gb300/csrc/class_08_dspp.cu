// (ds|pp) derivative-ERI class kernel instance.
#include "eri_fock.cuh"

namespace tg {

cudaError_t launch_qc08(int fp32, int grid, size_t smem, cudaStream_t st, const MolDesc *mols,
                         const ClassLaunch &cl, const OutArgs &out, const double *boys)
{
    return launch_class_kernel<2, 0, 1, 1>(fp32, grid, smem, st, mols, cl, out, boys);
}

cudaError_t launch_fock_qc08(int grid, cudaStream_t st, const MolDesc *mols, const ClassLaunch &cl,
                             const OutArgs &out, const double *boys)
{
    return launch_fock_class<2, 0, 1, 1>(grid, st, mols, cl, out, boys);
}

}  // namespace tg
