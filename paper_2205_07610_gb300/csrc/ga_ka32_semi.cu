// Inter-sequence kernel instantiations: CellS32, semi mode.
#include "ga_launch.h"

namespace ga {
GA_KA_DEFINE(ka32_semi, CellS32, kModeSemi)
}  // namespace ga
