// One instantiation set of the persistent kernels, chosen at compile time.  The build
// compiles this file once per precision mode (GTQA_UNIT_MODE = ModeFP64 | ModeMixed) and
// unit (GTQA_UNIT = 0 gates with the marginals, residual and sampling kernels, 1 BP,
// 2 regauge, 3 arbitrary gates), so the eight sets compile in parallel.
#include "gtqa_units.cuh"

#if !defined(GTQA_UNIT_MODE) || !defined(GTQA_UNIT)
#error "compile with -DGTQA_UNIT_MODE=<ModeFP64|ModeMixed> -DGTQA_UNIT=<0|1|2|3>"
#endif

namespace gtqa {

#if GTQA_UNIT == 0
template struct PhaseUnit<GTQA_UNIT_MODE, PK_GATES>;
template struct AuxUnit<GTQA_UNIT_MODE>;
#elif GTQA_UNIT == 1
template struct PhaseUnit<GTQA_UNIT_MODE, PK_BP>;
#elif GTQA_UNIT == 2
template struct PhaseUnit<GTQA_UNIT_MODE, PK_REGAUGE>;
#elif GTQA_UNIT == 3
template struct GeneralUnit<GTQA_UNIT_MODE>;
#else
#error "GTQA_UNIT must be 0, 1, 2 or 3"
#endif

}  // namespace gtqa
