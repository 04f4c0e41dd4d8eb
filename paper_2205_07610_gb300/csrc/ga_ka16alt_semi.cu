// Packed inter-sequence tiles with the alternative lane-group size, semi mode.
#include "ga_launch.h"

namespace ga {
GA_KA_ALT_DEFINE(ka16alt_semi, kModeSemi)
}  // namespace ga
