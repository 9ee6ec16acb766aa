// chain_b.cu -- C0 chains with the de Casteljau and Seiler evaluators.
#include "chain_eval.cuh"

namespace bez {
LaunchResult launch_chain_decasteljau(const CurveArgs& a, int tm, int om, cudaStream_t s, const LaunchHooks& h)
{
    return launch_chain_variant<VAR_DECASTELJAU>(a, tm, om, s, h);
}
LaunchResult launch_chain_seiler(const CurveArgs& a, int tm, int om, cudaStream_t s, const LaunchHooks& h)
{
    return launch_chain_variant<VAR_SEILER>(a, tm, om, s, h);
}
}  // namespace bez
