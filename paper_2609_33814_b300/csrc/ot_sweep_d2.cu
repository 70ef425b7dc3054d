// Instantiations of the sweep kernel for d = 2.
#include "ot_sweep.cuh"

namespace ot {

SweepFn get_sweep_d2(int mode, int R, int ch, int v) { return sweep_m<2>(mode, R, ch, v); }

}  // namespace ot
