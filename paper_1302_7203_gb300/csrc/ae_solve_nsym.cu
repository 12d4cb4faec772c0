// ae_solve_nsym.cu -- the pipeline of ae_solve.cuh instantiated for
// non-symmetric arrowheads (Remark of Sec. 6.1).
#include "ae_solve.cuh"

namespace ae {

void launch_pipeline_nsym(int n, int grid, Scratch S, const SolveOpts &so, const RunOpts &ro,
                          const VecArgs &va, cudaStream_t st) {
    launch_pipeline<KIND_ARROW, KIND_NSYM>(n, grid, S, so, ro, va, st);
}

}  // namespace ae
