// ae_solve_herm.cu -- the pipeline of ae_solve.cuh instantiated for
// Hermitian arrowheads (Sec. 6.1).
#include "ae_solve.cuh"

namespace ae {

void launch_pipeline_herm(int n, int grid, Scratch S, const SolveOpts &so, const RunOpts &ro,
                          const VecArgs &va, cudaStream_t st) {
    launch_pipeline<KIND_ARROW, KIND_HERM>(n, grid, S, so, ro, va, st);
}

}  // namespace ae
