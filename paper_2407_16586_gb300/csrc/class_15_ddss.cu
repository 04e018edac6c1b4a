// (dd|ss) derivative-ERI class kernel instance.
#include "eri_warp.cuh"

namespace tg {

cudaError_t launch_qc15(int fp32, int grid, size_t smem, cudaStream_t st, const MolDesc *mols,
                         const ClassLaunch &cl, const OutArgs &out, const double *boys)
{
    return launch_class_kernel<2, 2, 0, 0>(fp32, grid, smem, st, mols, cl, out, boys);
}

}  // namespace tg
