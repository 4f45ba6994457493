// An application the paper does not have, added through the vertex-program
// interface alone (include/ipregel_program.cuh), with no change to the engine:
// the most reliable path from a source. Each edge carries a survival probability
// p(u,v) = w(u,v) / 256 (the graph's uint32 weights, 1..255; weight 1 for an
// unweighted graph); a vertex's value is the largest product of probabilities
// over the paths from the source, the product taken in FP32 along the path from
// the source outwards. Max over float products has no hardware atomic, so the
// push exchange combines with the compare-and-swap loop of combine_atomic.
#include "engine.cuh"

struct ReliabilityProgram {
    using Combiner = ipregel::MaxCombiner<float>;  // no hardware float atomicMax: CAS loop
    using Value = float;
    static constexpr bool kWeighted = true;
    static constexpr bool kAllBroadcastAtStart = false;
    static constexpr bool kUsesSource = true;
    static constexpr bool kEarlyExitUnweighted = false;
    static constexpr bool kBlockedMinPull = false;
    // superstep 0: the source is certain (1) and broadcasts; every other vertex 0
    __device__ static bool init(uint32_t v, uint32_t, uint32_t source, Value& value) {
        value = v == source ? 1.0f : 0.0f;
        return v == source;
    }
    // w * 2^-8 is exact in FP32 for w < 2^24; one rounded product per edge
    __device__ static Value message(Value value, uint32_t w) { return value * ((float)w * 0.00390625f); }
    __device__ static bool compute(Value& value, Value combined) {
        if (combined > value) {
            value = combined;
            return true;
        }
        return false;
    }
};

static_assert(!ipregel::has_hw_atomic<ReliabilityProgram::Combiner>::value, "float max combines by CAS");
static_assert(ipregel::has_hw_atomic<ipregel::MinCombiner<uint32_t>>::value, "uint32 min is atomicMin");

IPG_REGISTER_PROGRAM(ReliabilityProgram, IP_RELIABILITY)
