// Inter-sequence kernel instantiations: CellS16x2, global mode.
#include "ga_launch.h"

namespace ga {
GA_KA_DEFINE(ka16_global, CellS16x2, kModeGlobal)
}  // namespace ga
