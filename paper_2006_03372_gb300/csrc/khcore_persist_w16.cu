// khcore_persist_w16.cu — persistent decomposition kernel for W = 16
// (64*16 sources per BFS batch); one translation unit per W so that the
// variants compile in parallel.
#include "khcore_persist.cuh"

namespace khc {
cudaError_t persist_launch_16(const PersistLaunch &L, int grid, cudaStream_t s) { return persist_launch_w<16, 1>(L, grid, s); }
int persist_occupancy_16() { return persist_occupancy_w<16, 1>(); }
}  // namespace khc
