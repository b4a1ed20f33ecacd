// khcore_persist_w4.cu — persistent decomposition kernel for W = 4
// (64*4 sources per BFS batch); one translation unit per W so that the
// variants compile in parallel.
#include "khcore_persist.cuh"

namespace khc {
cudaError_t persist_launch_4(const PersistLaunch &L, int grid, cudaStream_t s) { return persist_launch_w<4, 1>(L, grid, s); }
int persist_occupancy_4() { return persist_occupancy_w<4, 1>(); }
}  // namespace khc
