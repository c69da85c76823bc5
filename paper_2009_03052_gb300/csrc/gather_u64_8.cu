// gather_u64_8.cu -- instantiations of the neighbour-sum kernel for
// u64 counts in 8-byte units (kept in a translation unit of
// their own so the build compiles them in parallel).
#include "gather.cuh"

namespace mc {

GatherKernel gather_kernel_ptr_u64_8(int G, int NU, int U, int MB)
{
#define MC_G(G_, NU_, U_, MB_) \
    if (G == G_ && NU == NU_ && U == U_ && MB == MB_) return gather_kernel<uint64_t, 8, G_, NU_, U_, MB_>;
    MC_G(1, 1, 8, 1)
    MC_G(1, 1, 4, 1)
    MC_G(1, 1, 2, 1)
    MC_G(1, 1, 4, 6)
    MC_G(1, 1, 2, 8)
    MC_G(1, 1, 1, 8)
    MC_G(2, 1, 8, 1)
    MC_G(2, 1, 4, 1)
    MC_G(2, 1, 2, 1)
    MC_G(2, 1, 4, 6)
    MC_G(2, 1, 2, 8)
    MC_G(2, 1, 1, 8)
    MC_G(4, 1, 8, 1)
    MC_G(4, 1, 4, 1)
    MC_G(4, 1, 2, 1)
    MC_G(4, 1, 4, 6)
    MC_G(4, 1, 2, 8)
    MC_G(4, 1, 1, 8)
    MC_G(8, 1, 8, 1)
    MC_G(8, 1, 4, 1)
    MC_G(8, 1, 2, 1)
    MC_G(8, 1, 4, 6)
    MC_G(8, 1, 2, 8)
    MC_G(8, 1, 1, 8)
    MC_G(16, 1, 8, 1)
    MC_G(16, 1, 4, 1)
    MC_G(16, 1, 2, 1)
    MC_G(16, 1, 4, 6)
    MC_G(16, 1, 2, 8)
    MC_G(16, 1, 1, 8)
    MC_G(32, 1, 8, 1)
    MC_G(32, 1, 4, 1)
    MC_G(32, 1, 2, 1)
    MC_G(32, 1, 4, 6)
    MC_G(32, 1, 2, 8)
    MC_G(32, 1, 1, 8)
    MC_G(32, 2, 8, 1)
    MC_G(32, 2, 4, 1)
    MC_G(32, 2, 2, 1)
    MC_G(32, 2, 4, 6)
    MC_G(32, 2, 2, 8)
    MC_G(32, 2, 1, 8)
    MC_G(32, 4, 4, 1)
    MC_G(32, 4, 2, 1)
    MC_G(32, 4, 1, 1)
    MC_G(32, 4, 2, 6)
    MC_G(32, 4, 1, 8)
    MC_G(32, 8, 2, 1)
    MC_G(32, 8, 1, 1)
    MC_G(32, 8, 1, 6)
    MC_G(32, 8, 1, 8)
    MC_G(32, 16, 1, 1)
    MC_G(32, 16, 1, 6)
    MC_G(32, 16, 1, 8)
    MC_G(1, 2, 2, 8)
    MC_G(2, 2, 2, 8)
    MC_G(4, 2, 2, 8)
    MC_G(8, 2, 2, 8)
#undef MC_G
    return nullptr;
}

}  // namespace mc
