// khcore_persist_w8.cu — persistent decomposition kernel for W = 8
// (64*8 sources per BFS batch); one translation unit per W so that the
// variants compile in parallel.
#include "khcore_persist.cuh"

namespace khc {
cudaError_t persist_launch_8(const PersistLaunch &L, int grid, cudaStream_t s) { return persist_launch_w<8, 1>(L, grid, s); }
int persist_occupancy_8() { return persist_occupancy_w<8, 1>(); }
}  // namespace khc
