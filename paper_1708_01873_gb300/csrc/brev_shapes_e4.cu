// Tile kernels for 4-byte elements (float32, uint32).
#include "brev_kernels.cuh"

namespace brev {
const ShapeEntry g_shapes_e4[] = {
    // 16-byte vector path
    BREV_OOP2(4, 5, 5), BREV_OOP2(4, 6, 6), BREV_OOP2(4, 7, 7),
    BREV_OOP2(4, 5, 6), BREV_OOP2(4, 6, 5), BREV_OOP2(4, 6, 7),
    BREV_OOP2(4, 7, 6),
    BREV_INP2(4, 5),    BREV_INP2(4, 6),    BREV_INP2(4, 7),
    // element-wide path (pointers aligned to 4 but not 16 bytes)
    BREV_OOP(4, 4, 5, 5),  BREV_OOP(4, 4, 6, 6),
    BREV_INP(4, 4, 5),     BREV_INP(4, 4, 6),
};
const int g_shapes_e4_n = sizeof(g_shapes_e4) / sizeof(g_shapes_e4[0]);
}  // namespace brev
