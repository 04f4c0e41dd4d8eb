// Inter-sequence kernel instantiations: CellS32, global mode.
#include "ga_launch.h"

namespace ga {
GA_KA_DEFINE(ka32_global, CellS32, kModeGlobal)
}  // namespace ga
