// Tile kernels for 16-byte elements (complex<double>).
#include "brev_kernels.cuh"

namespace brev {
const ShapeEntry g_shapes_e16[] = {
    BREV_OOP2(16, 3, 3), BREV_OOP2(16, 4, 4), BREV_OOP2(16, 5, 5),
    BREV_OOP2(16, 6, 6), BREV_OOP2(16, 4, 5), BREV_OOP2(16, 5, 4),
    BREV_OOP2(16, 5, 6), BREV_OOP2(16, 6, 5),
    BREV_INP2(16, 3),    BREV_INP2(16, 4),    BREV_INP2(16, 5),
    BREV_INP2(16, 6),
};
const int g_shapes_e16_n = sizeof(g_shapes_e16) / sizeof(g_shapes_e16[0]);
}  // namespace brev
