// khcore_persist_w2.cu — persistent decomposition kernel for W = 2
// (64*2 sources per BFS batch); one translation unit per W so that the
// variants compile in parallel.
#include "khcore_persist.cuh"

namespace khc {
cudaError_t persist_launch_2(const PersistLaunch &L, int grid, cudaStream_t s) { return persist_launch_w<2, 1>(L, grid, s); }
int persist_occupancy_2() { return persist_occupancy_w<2, 1>(); }
}  // namespace khc
