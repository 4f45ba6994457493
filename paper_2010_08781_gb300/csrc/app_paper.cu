// The paper's two min-combiner applications written as vertex programs
// (include/ipregel_program.cuh) and registered with the engine.
#include "engine.cuh"

// Hashmin connected components, Fig. 9: superstep 0 takes the vertex's id as its
// label and broadcasts it; later, a smaller combined label replaces the label and
// is broadcast. The id is the caller's id when the library renumbered the graph.
struct HashminProgram {
    using Combiner = ipregel::MinCombiner<uint32_t>;  // Fig. 5's min combiner: atomicMin
    using Value = uint32_t;
    static constexpr bool kWeighted = false;
    static constexpr bool kAllBroadcastAtStart = true;
    static constexpr bool kUsesSource = false;
    static constexpr bool kEarlyExitUnweighted = false;
    static constexpr bool kBlockedMinPull = true;  // message = value, labels < 2^32 - 1
    __device__ static bool init(uint32_t, uint32_t caller_id, uint32_t, Value& value) {
        value = caller_id;
        return true;
    }
    __device__ static Value message(Value value, uint32_t) { return value; }
    __device__ static bool compute(Value& value, Value combined) {
        if (combined < value) {
            value = combined;
            return true;
        }
        return false;
    }
};

// Single-source shortest paths, Fig. 10 with per-edge weights: the source starts
// at 0 and broadcasts, every other vertex at "infinity" (0xFFFFFFFF); the message
// along an edge is the distance plus the edge's weight, saturating at infinity.
// With unit weights every broadcaster of a superstep holds the same distance,
// which allows the early-exit pull.
struct SsspProgram {
    using Combiner = ipregel::MinCombiner<uint32_t>;
    using Value = uint32_t;
    static constexpr bool kWeighted = true;
    static constexpr bool kAllBroadcastAtStart = false;
    static constexpr bool kUsesSource = true;
    static constexpr bool kEarlyExitUnweighted = true;
    static constexpr bool kBlockedMinPull = false;  // the message reads the edge weight,
    static constexpr bool kBlockedMinPullAddsWeight = true;  // and adds it: a broadcast distance is a
                                                             // path's length, at most (V - 1) x max weight
    __device__ static bool init(uint32_t v, uint32_t, uint32_t source, Value& value) {
        value = v == source ? 0u : 0xFFFFFFFFu;
        return v == source;
    }
    __device__ static Value message(Value value, uint32_t w) {
        const uint32_t s = value + w;
        return s < value ? 0xFFFFFFFFu : s;
    }
    __device__ static bool compute(Value& value, Value combined) {
        if (combined < value) {
            value = combined;
            return true;
        }
        return false;
    }
};

IPG_REGISTER_PROGRAM(HashminProgram, IP_HASHMIN)
IPG_REGISTER_PROGRAM(SsspProgram, IP_SSSP)
