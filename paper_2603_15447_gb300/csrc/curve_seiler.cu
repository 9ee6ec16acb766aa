// curve_seiler.cu -- instantiates the seiler register evaluator (see curve_eval.cuh).
#include "curve_eval.cuh"

namespace bez {
LaunchResult launch_curve_seiler(const CurveArgs& a, int tm, int om, cudaStream_t s, const LaunchHooks& h)
{
    return launch_curve_variant<VAR_SEILER>(a, tm, om, s, h);
}
}  // namespace bez
