// khcore_persist_w4x2.cu — persistent decomposition kernel for W = 4 with two
// resident blocks per SM (64 registers per thread); one translation unit per
// variant so that they compile in parallel.
#include "khcore_persist.cuh"

namespace khc {
cudaError_t persist_launch_4x2(const PersistLaunch &L, int grid, cudaStream_t s)
{
    return persist_launch_w<4, 2>(L, grid, s);
}
int persist_occupancy_4x2() { return persist_occupancy_w<4, 2>(); }
}  // namespace khc
