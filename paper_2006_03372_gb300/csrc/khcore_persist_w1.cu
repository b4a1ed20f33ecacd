// khcore_persist_w1.cu — persistent decomposition kernel for W = 1
// (64*1 sources per BFS batch); one translation unit per W so that the
// variants compile in parallel.
#include "khcore_persist.cuh"

namespace khc {
cudaError_t persist_launch_1(const PersistLaunch &L, int grid, cudaStream_t s) { return persist_launch_w<1, 1>(L, grid, s); }
int persist_occupancy_1() { return persist_occupancy_w<1, 1>(); }
}  // namespace khc
