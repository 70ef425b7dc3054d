// Instantiations of the sweep kernel for d = 1.
#include "ot_sweep.cuh"

namespace ot {

SweepFn get_sweep_d1(int mode, int R, int ch, int v) { return sweep_m<1>(mode, R, ch, v); }

}  // namespace ot
