// ae_solve_dpr1.cu -- the pipeline of ae_solve.cuh instantiated for
// DPR1 matrices D + rho u u^T (Sec. 6.3).
#include "ae_solve.cuh"

namespace ae {

void launch_pipeline_dpr1(int n, int grid, Scratch S, const SolveOpts &so, const RunOpts &ro,
                          const VecArgs &va, cudaStream_t st) {
    launch_pipeline<KIND_DPR1, KIND_DPR1>(n, grid, S, so, ro, va, st);
}

}  // namespace ae
