// ae_solve_svd.cu -- the pipeline of ae_solve.cuh instantiated for
// the SVD of a triangular arrowhead (Sec. 6.2).
#include "ae_solve.cuh"

namespace ae {

void launch_pipeline_tsvd(int n, int grid, Scratch S, const SolveOpts &so, const RunOpts &ro,
                          const VecArgs &va, cudaStream_t st) {
    launch_pipeline<KIND_TSVD, KIND_TSVD>(n, grid, S, so, ro, va, st);
}

}  // namespace ae
