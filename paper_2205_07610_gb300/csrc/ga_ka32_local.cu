// Inter-sequence kernel instantiations: CellS32, local mode.
#include "ga_launch.h"

namespace ga {
GA_KA_DEFINE(ka32_local, CellS32, kModeLocal)
}  // namespace ga
