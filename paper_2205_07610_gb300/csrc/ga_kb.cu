// Long-pair (multi-stage) kernel instantiations: every mode, selector and
// profile substitution paths.
#include "ga_launch.h"

namespace ga {
GA_KB_DEFINE(kb_local_sel, kModeLocal, false)
GA_KB_DEFINE(kb_global_sel, kModeGlobal, false)
GA_KB_DEFINE(kb_semi_sel, kModeSemi, false)
GA_KB_DEFINE(kb_local_prof, kModeLocal, true)
GA_KB_DEFINE(kb_global_prof, kModeGlobal, true)
GA_KB_DEFINE(kb_semi_prof, kModeSemi, true)
}  // namespace ga
