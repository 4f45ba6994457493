/*
 * ipregel_program.cuh — the vertex-centric programming interface of
 * libipregel_gb300 (C++ / CUDA, sm_103a).
 *
 * The paper's user interface (Section 4.1, Figs. 1 and 2) is a compute()
 * function run by every active vertex in every superstep, plus a combine()
 * function that folds two messages for the same recipient into one (Section
 * 4.3.3). The GPU engine runs that model with the exchange, selection, halting
 * and scheduling machinery of the library; a program supplies only the
 * per-vertex arithmetic, as a struct of static device functions:
 *
 *   struct MyProgram {
 *     using Combiner = ipregel::MinCombiner<uint32_t>;   // or Max / Sum / a custom one
 *     using Value = typename Combiner::T;                 // 32-bit vertex value = message type
 *     static constexpr bool kWeighted = ...;              // message() reads the edge weight
 *     static constexpr bool kAllBroadcastAtStart = ...;   // init() returns true for every vertex
 *     static constexpr bool kUsesSource = ...;            // init() reads the run's source vertex
 *     static constexpr bool kEarlyExitUnweighted = ...;   // on an unweighted graph every message
 *                                                         // into a superstep is the same (a pull may
 *                                                         // stop at the first one)
 *     static constexpr bool kBlockedMinPull = ...;        // Combiner is MinCombiner<uint32_t>, message()
 *                                                         // returns the value unchanged and never the
 *                                                         // all-ones pattern: the pull may stream the
 *                                                         // blocked edge layout (Hashmin)
 *     // optional (false when absent):
 *     static constexpr bool kBlockedMinPullAddsWeight = ...;  // Combiner is MinCombiner<uint32_t>,
 *                                                         // message(value, w) is value + w and every value
 *                                                         // the program broadcasts is at most (V - 1) times
 *                                                         // the largest weight: the pull may stream the
 *                                                         // blocked layout with the weights stored there as
 *                                                         // one byte per edge, on graphs whose weights are
 *                                                         // below 256 and V times the largest weight below
 *                                                         // 2^32 - 1, so that no message reaches the
 *                                                         // all-ones pattern (SSSP)
 *     // superstep 0 (the first superstep, Section 4.3.1 condition 1): set the initial
 *     // value and return whether the vertex broadcasts it (caller_id: the vertex's id
 *     // in the caller's numbering; source: ip_options_t.source in the internal one)
 *     __device__ static bool init(uint32_t v, uint32_t caller_id, uint32_t source, Value& value);
 *     // the message sent along an out-edge with weight w (1 for unweighted graphs)
 *     __device__ static Value message(Value value, uint32_t w);
 *     // superstep >= 1 for a vertex that received messages (their combination):
 *     // update the value, return true to broadcast the new value; the vertex then
 *     // votes to halt (Fig. 2's vote_to_halt), a new message re-activates it
 *     __device__ static bool compute(Value& value, Value combined);
 *   };
 *
 * A program never broadcasts the bit pattern kNoBroadcastBits (all ones; a NaN
 * for float values): the broadcast slot of a silent vertex holds it.
 *
 * This "improve and broadcast" shape is the one of Fig. 9 (Hashmin) and Fig. 10
 * (SSSP); the library's Hashmin and SSSP are written as such programs, and so
 * is an application the paper does not have (the most reliable path, a max
 * combiner over float products). PageRank (Fig. 8: every vertex active for T
 * supersteps, a sum combiner) keeps its own pull engines but its compute() and
 * its combiner come from this header too.
 *
 * Combiners and their atomics. The push exchange combines concurrent messages
 * into one mailbox slot. The paper locks the slot (Section 4.3.2) and leaves
 * lock-free combiners as future work (Section 9); here the combiner is chosen
 * at compile time: a MinCombiner / MaxCombiner / SumCombiner over a type with a
 * hardware atomic for that operation (min/max: 32-bit integers; sum: 32-bit
 * integers and float) maps to that atomic; any other combiner — a custom struct
 * with T, identity() and op(), or min/max over float — runs a compare-and-swap
 * loop on the slot's 32-bit word that applies op(). ipregel::has_hw_atomic<C>
 * tells which one a combiner gets.
 *
 * Register a program with the engine in a .cu file of the library:
 *     IPG_REGISTER_PROGRAM(MyProgram, app_id)
 * (app_id: the ip_app_t value ip_run() dispatches on; see csrc/app_*.cu).
 */
#ifndef IPREGEL_PROGRAM_CUH
#define IPREGEL_PROGRAM_CUH

#include <stdint.h>
#include <string.h>

#include <type_traits>

namespace ipregel {

// The broadcast slot of a vertex that did not broadcast holds this bit pattern;
// a program never broadcasts it (for float values it is a NaN).
constexpr uint32_t kNoBroadcastBits = 0xFFFFFFFFu;

template <class T>
__host__ __device__ __forceinline__ uint32_t to_bits(T x) {
    static_assert(sizeof(T) == 4, "vertex values and messages are 32-bit");
    uint32_t u;
    memcpy(&u, &x, 4);
    return u;
}
template <class T>
__host__ __device__ __forceinline__ T from_bits(uint32_t u) {
    T x;
    memcpy(&x, &u, 4);
    return x;
}
template <class T>
__host__ __device__ __forceinline__ T no_broadcast() {
    return from_bits<T>(kNoBroadcastBits);
}
template <class T>
__host__ __device__ __forceinline__ bool is_no_broadcast(T x) {
    return to_bits(x) == kNoBroadcastBits;
}

// ------------------------------------------------------------------ combiners
enum class CombineOp { kCustom, kMin, kMax, kSum };

template <class TT>
struct MinCombiner {
    using T = TT;
    static constexpr CombineOp kOp = CombineOp::kMin;
    __host__ __device__ static T identity() {
        if constexpr (std::is_floating_point<T>::value)
            return from_bits<T>(0x7F800000u);  // +infinity
        else if constexpr (std::is_signed<T>::value)
            return T(0x7FFFFFFF);
        else
            return T(0xFFFFFFFFu);
    }
    __host__ __device__ static T op(T a, T b) { return b < a ? b : a; }
    // a message that cannot change the slot need not be combined
    __host__ __device__ static bool improves(T msg, T cur) { return msg < cur; }
};

template <class TT>
struct MaxCombiner {
    using T = TT;
    static constexpr CombineOp kOp = CombineOp::kMax;
    __host__ __device__ static T identity() {
        if constexpr (std::is_floating_point<T>::value)
            return from_bits<T>(0xFF800000u);  // -infinity
        else if constexpr (std::is_signed<T>::value)
            return T(-2147483647 - 1);
        else
            return T(0);
    }
    __host__ __device__ static T op(T a, T b) { return b > a ? b : a; }
    __host__ __device__ static bool improves(T msg, T cur) { return msg > cur; }
};

template <class TT>
struct SumCombiner {
    using T = TT;
    static constexpr CombineOp kOp = CombineOp::kSum;
    __host__ __device__ static T identity() { return T(0); }
    __host__ __device__ static T op(T a, T b) { return a + b; }
    __host__ __device__ static bool improves(T, T) { return true; }
};

// A combiner that declares no kOp is custom: identity() and op() only.
template <class C, class = void>
struct op_of {
    static constexpr CombineOp value = CombineOp::kCustom;
};
template <class C>
struct op_of<C, std::void_t<decltype(C::kOp)>> {
    static constexpr CombineOp value = C::kOp;
};
template <class C, class = void>
struct has_improves : std::false_type {};
template <class C>
struct has_improves<C, std::void_t<decltype(C::improves(typename C::T(), typename C::T()))>> : std::true_type {};

// A program's optional kBlockedMinPullAddsWeight (false when it declares none).
template <class P, class = void>
struct blocked_pull_adds_weight : std::false_type {};
template <class P>
struct blocked_pull_adds_weight<P, std::void_t<decltype(P::kBlockedMinPullAddsWeight)>>
    : std::integral_constant<bool, P::kBlockedMinPullAddsWeight> {};

// Does this combiner map to one hardware atomic on sm_103a?
template <class C>
struct has_hw_atomic {
    using T = typename C::T;
    static constexpr CombineOp o = op_of<C>::value;
    static constexpr bool int32 = std::is_same<T, uint32_t>::value || std::is_same<T, int32_t>::value;
    static constexpr bool value = ((o == CombineOp::kMin || o == CombineOp::kMax) && int32) ||
                                  (o == CombineOp::kSum && (int32 || std::is_same<T, float>::value));
};

// Combines v into *slot. Hardware atomic where has_hw_atomic holds, otherwise a
// compare-and-swap loop on the slot's bits applying C::op (lock free: a thread
// retries only when another thread changed the slot in between).
template <class C>
__device__ __forceinline__ void combine_atomic(typename C::T* slot, typename C::T v) {
    using T = typename C::T;
    constexpr CombineOp o = op_of<C>::value;
    if constexpr (has_hw_atomic<C>::value) {
        if constexpr (o == CombineOp::kMin)
            atomicMin(slot, v);
        else if constexpr (o == CombineOp::kMax)
            atomicMax(slot, v);
        else
            atomicAdd(slot, v);
    } else {
        unsigned int* w = reinterpret_cast<unsigned int*>(slot);
        unsigned int old = *reinterpret_cast<volatile unsigned int*>(w);
        for (;;) {
            const T cur = from_bits<T>(old);
            const T nxt = C::op(cur, v);
            if (to_bits(nxt) == old) return;  // nothing to change
            const unsigned int seen = atomicCAS(w, old, to_bits(nxt));
            if (seen == old) return;
            old = seen;
        }
    }
}

// Whether a message may change a slot holding cur (a cheap read before the atomic).
template <class C>
__device__ __forceinline__ bool may_improve(typename C::T msg, typename C::T cur) {
    if constexpr (has_improves<C>::value)
        return C::improves(msg, cur);
    else
        return to_bits(C::op(cur, msg)) != to_bits(cur);
}

// Folds the 32 lanes' values with C::op; every lane gets the result.
template <class C>
__device__ __forceinline__ typename C::T warp_combine(typename C::T x) {
    using T = typename C::T;
    if constexpr (op_of<C>::value == CombineOp::kMin && std::is_same<T, uint32_t>::value) {
        return __reduce_min_sync(0xFFFFFFFFu, x);
    } else if constexpr (op_of<C>::value == CombineOp::kMax && std::is_same<T, uint32_t>::value) {
        return __reduce_max_sync(0xFFFFFFFFu, x);
    } else {
        for (int o = 16; o > 0; o >>= 1) x = C::op(x, from_bits<T>(__shfl_xor_sync(0xFFFFFFFFu, to_bits(x), o)));
        return x;
    }
}

}  // namespace ipregel

#endif  // IPREGEL_PROGRAM_CUH
