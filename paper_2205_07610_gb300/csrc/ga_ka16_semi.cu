// Inter-sequence kernel instantiations: CellS16x2, semi mode.
#include "ga_launch.h"

namespace ga {
GA_KA_DEFINE(ka16_semi, CellS16x2, kModeSemi)
}  // namespace ga
