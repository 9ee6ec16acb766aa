// curve_bernstein.cu -- instantiates the bernstein register evaluator (see curve_eval.cuh).
#include "curve_eval.cuh"

namespace bez {
LaunchResult launch_curve_bernstein(const CurveArgs& a, int tm, int om, cudaStream_t s, const LaunchHooks& h)
{
    return launch_curve_variant<VAR_BERNSTEIN>(a, tm, om, s, h);
}
}  // namespace bez
