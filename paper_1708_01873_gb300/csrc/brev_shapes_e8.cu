// Tile kernels for 8-byte elements (complex<float>, double, uint64).
#include "brev_kernels.cuh"

namespace brev {
const ShapeEntry g_shapes_e8[] = {
    // 16-byte vector path
    BREV_OOP2(8, 4, 4), BREV_OOP2(8, 5, 5), BREV_OOP2(8, 6, 6),
    BREV_OOP2(8, 4, 5), BREV_OOP2(8, 5, 4), BREV_OOP2(8, 5, 6),
    BREV_OOP2(8, 6, 5),
    BREV_INP2(8, 4),    BREV_INP2(8, 5),    BREV_INP2(8, 6),
    // element-wide path (pointers aligned to 8 but not 16 bytes)
    BREV_OOP(8, 8, 4, 4),  BREV_OOP(8, 8, 5, 5),
    BREV_INP(8, 8, 4),     BREV_INP(8, 8, 5),
};
const int g_shapes_e8_n = sizeof(g_shapes_e8) / sizeof(g_shapes_e8[0]);
}  // namespace brev
