// chain_a.cu -- C0 chains with the power-basis and Bernstein evaluators.
#include "chain_eval.cuh"

namespace bez {
LaunchResult launch_chain_horner(const CurveArgs& a, int tm, int om, cudaStream_t s, const LaunchHooks& h)
{
    return launch_chain_variant<VAR_HORNER>(a, tm, om, s, h);
}
LaunchResult launch_chain_horner_centred(const CurveArgs& a, int tm, int om, cudaStream_t s, const LaunchHooks& h)
{
    return launch_chain_variant<VAR_HORNER_CENTRED>(a, tm, om, s, h);
}
LaunchResult launch_chain_bernstein(const CurveArgs& a, int tm, int om, cudaStream_t s, const LaunchHooks& h)
{
    return launch_chain_variant<VAR_BERNSTEIN>(a, tm, om, s, h);
}
}  // namespace bez
