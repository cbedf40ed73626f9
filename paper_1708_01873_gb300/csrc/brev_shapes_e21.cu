// Tile kernels for 2- and 1-byte elements, and the small-array kernels.
#include "brev_kernels.cuh"

namespace brev {
const ShapeEntry g_shapes_e21[] = {
    BREV_OOP2(2, 6, 6), BREV_OOP2(2, 7, 7),
    BREV_INP2(2, 6),    BREV_INP2(2, 7),
    BREV_OOP(2, 2, 6, 6),  BREV_INP(2, 2, 6),
    BREV_OOP2(1, 7, 7), BREV_OOP2(1, 8, 8),
    BREV_INP2(1, 7),    BREV_INP2(1, 8),
    BREV_OOP(1, 1, 7, 7),  BREV_INP(1, 1, 7),
};
const int g_shapes_e21_n = sizeof(g_shapes_e21) / sizeof(g_shapes_e21[0]);

const void* small_kernel(int E) {
  switch (E) {
    case 1: return (const void*)&k_small<1>;
    case 2: return (const void*)&k_small<2>;
    case 4: return (const void*)&k_small<4>;
    case 8: return (const void*)&k_small<8>;
    case 16: return (const void*)&k_small<16>;
    default: return nullptr;
  }
}
}  // namespace brev
