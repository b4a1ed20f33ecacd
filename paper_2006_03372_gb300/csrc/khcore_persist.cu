// khcore_persist.cu — dispatch of the persistent decomposition kernel by W.
#include "khcore_persist.cuh"

namespace khc {

cudaError_t launch_decompose_persist(int W, const PersistLaunch &L, int grid, cudaStream_t s, int minb)
{
    switch (W) {
    case 1: return persist_launch_1(L, grid, s);
    case 2: return persist_launch_2(L, grid, s);
    case 4: return minb == 2 ? persist_launch_4x2(L, grid, s) : persist_launch_4(L, grid, s);
    case 8: return persist_launch_8(L, grid, s);
    case 16: return persist_launch_16(L, grid, s);
    default: return cudaErrorInvalidValue;
    }
}

int max_blocks_per_sm_persist(int W, int minb)
{
    switch (W) {
    case 1: return persist_occupancy_1();
    case 2: return persist_occupancy_2();
    case 4: return minb == 2 ? persist_occupancy_4x2() : persist_occupancy_4();
    case 8: return persist_occupancy_8();
    case 16: return persist_occupancy_16();
    default: return 0;
    }
}

}  // namespace khc
