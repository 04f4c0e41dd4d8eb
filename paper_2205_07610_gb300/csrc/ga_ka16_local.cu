// Inter-sequence kernel instantiations: CellS16x2, local mode.
#include "ga_launch.h"

namespace ga {
GA_KA_DEFINE(ka16_local, CellS16x2, kModeLocal)
}  // namespace ga
