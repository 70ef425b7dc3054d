// Instantiations of the sweep kernel for d = 3.
#include "ot_sweep.cuh"

namespace ot {

SweepFn get_sweep_d3(int mode, int R, int ch, int v) { return sweep_m<3>(mode, R, ch, v); }

}  // namespace ot
