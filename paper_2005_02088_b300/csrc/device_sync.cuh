// Device synchronisation primitives of the Camelot pipeline runtime.
//
// The global-memory handoff (Sec. 6.2) is a sequence flag per ring slot written
// with release semantics by the producer and read with acquire semantics by
// the consumer; everything the producer wrote before the release is then
// visible to the consumer, which reads the slot in place.  Stage instances
// (the N_i x p_i SM partitions of Eq. 1) are groups of CTAs of one cooperative
// persistent kernel; a group synchronises through a counter barrier in global
// memory.  Every wait here is bounded: it gives up at a %globaltimer deadline
// (and after an iteration cap, should the timer stall), records an error code
// in the pipeline's status word and returns false; callers then unwind and
// the kernel exits, leaving the GPU usable.
#pragma once
#include <cstdint>

namespace camelot {

// Error codes the device writes into Ctl::status (first error wins).
enum DevError : uint32_t {
    DEV_OK = 0,
    DEV_ERR_GROUP_BARRIER = 1,   // an instance's CTAs did not all arrive in time
    DEV_ERR_OUT_SLOT = 2,        // no free output slot in time (downstream stalled)
    DEV_ERR_MAILBOX = 3,         // a CTA waited too long for its leader
    DEV_ERR_BAD_BATCH = 4,       // inconsistent batch descriptor
};

struct alignas(128) Line64 {
    unsigned long long v;
    unsigned long long pad[15];
};

// Control block of one pipeline in device memory.
struct alignas(128) Ctl {
    Line64 in_head;                  // next query ticket the batch trigger will take
    Line64 status;                   // DevError (low 32 bits) | where << 32
    Line64 trace_t0;                 // device time the running trace started (0 = not yet)
    Line64 exited[8];                // instances of stage s that have exited this launch
    Line64 batches[8];               // batches finished by stage s (statistics)
    Line64 busy_ns[8];               // stage s: summed over its batches, the time from the
                                     // instance holding its work to the batch published
    Line64 body_ns[8];               // stage s: summed over its batches, the time the
                                     // leader CTA spent in the stage body itself
    Line64 acq_ns[8];                // stage s: summed over its batches, the time its
                                     // leaders spent finding each batch's work
};

// Flags the host writes and the device reads (pinned, mapped host memory).
struct alignas(128) HostFlags {
    volatile unsigned long long stop;   // host asks the kernel to exit
    unsigned long long pad[15];
};

__device__ __forceinline__ uint64_t gtime() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint64_t ld_acquire_gpu(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ uint32_t ld_acquire_gpu32(const unsigned int* p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_gpu(unsigned long long* p, unsigned long long v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void st_release_gpu32(unsigned int* p, unsigned int v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
// System-scope forms, for words in pinned host memory (generic addressing).
__device__ __forceinline__ uint64_t ld_acquire_sys(const volatile unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.sys.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_sys(volatile unsigned long long* p, unsigned long long v) {
    asm volatile("st.release.sys.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ uint64_t ld_relaxed_gpu(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void record_error(Ctl* ctl, uint32_t code, uint32_t where) {
    unsigned long long w = (unsigned long long)code | ((unsigned long long)where << 32);
    atomicCAS(&ctl->status.v, 0ull, w);
}
__device__ __forceinline__ bool has_error(const Ctl* ctl) {
    return ld_relaxed_gpu(&ctl->status.v) != 0ull;
}

// Bounded back-off: returns false once `deadline` passed or `iters` ran out.
// The first 16 steps only re-check (hand-offs inside a running batch finish
// within a few hundred nanoseconds); later steps sleep 32, 64, ... 256 ns.
struct Backoff {
    uint64_t deadline;
    uint64_t iters_left;
    unsigned ns;
    unsigned n;
    __device__ explicit Backoff(uint64_t limit_ns)
        : deadline(gtime() + limit_ns), iters_left(limit_ns / 16 + 4000000ull), ns(32), n(0) {}
    __device__ __forceinline__ bool step() {
        if (--iters_left == 0) return false;
        if (gtime() > deadline) return false;
        if (++n > 16) {
            __nanosleep(ns);
            ns = ns < 256 ? ns * 2 : 256;
        }
        return true;
    }
    // true on every 16th step: for checks too costly to make on every one
    __device__ __forceinline__ bool sparse() const { return (n & 15u) == 0; }
};

// Barrier over the `nctas` CTAs of one stage instance.  All threads of every
// CTA call it.  Writes made by any thread before the barrier are visible to
// every thread of the group after it.  Returns false on timeout or on a
// pipeline error (then every caller must unwind).
struct alignas(128) GroupSync {
    unsigned int arrive;
    unsigned int pad0[31];
    unsigned int gen;
    unsigned int pad1[31];
    unsigned int done;               // running count: batches finished by each non-leader CTA, summed
    unsigned int pad_d[31];
    // mailbox: the leader fills it, then releases mb_gen = batch number + 1
    unsigned int cmd;
    unsigned int n;
    unsigned int from_trace;
    unsigned int mb_gen;
    unsigned long long in_ticket;    // input slot ticket (stage s >= 1)
    unsigned long long out_ticket;   // output slot ticket (non-final stages)
    unsigned long long first;        // first query ticket of the batch
    long long t_batch;
    unsigned int pad3[20];
};

__device__ __forceinline__ bool group_barrier(GroupSync* g, int nctas, Ctl* ctl,
                                              uint64_t limit_ns, uint32_t where,
                                              uint32_t err = DEV_ERR_GROUP_BARRIER) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        if (nctas > 1) {
            unsigned int my_gen = *(volatile unsigned int*)&g->gen;
            __threadfence();
            unsigned int arrived = atomicAdd(&g->arrive, 1u);
            if (arrived == (unsigned)nctas - 1u) {
                atomicExch(&g->arrive, 0u);
                __threadfence();
                st_release_gpu32(&g->gen, my_gen + 1u);
            } else {
                Backoff bo(limit_ns);
                while (ld_acquire_gpu32(&g->gen) == my_gen) {
                    if ((bo.sparse() && has_error(ctl)) || !bo.step()) {
                        record_error(ctl, err, where);
                        ok = 0;
                        break;
                    }
                }
            }
            __threadfence();
        }
        s_ok = ok && !has_error(ctl);
    }
    __syncthreads();
    return s_ok != 0;
}

// Bounded wait (one thread) until the 32-bit word at p equals v, read with
// acquire semantics; records `err` at `where` and returns false on timeout or
// on a pipeline error.
__device__ __forceinline__ bool wait_eq32(const unsigned int* p, unsigned int v, Ctl* ctl, uint64_t limit_ns,
                                          uint32_t where, uint32_t err) {
    if (ld_acquire_gpu32(p) == v) return true;
    Backoff bo(limit_ns);
    while (ld_acquire_gpu32(p) != v) {
        if ((bo.sparse() && has_error(ctl)) || !bo.step()) {
            record_error(ctl, err, where);
            return false;
        }
    }
    return true;
}

// 16-byte store of two 8-byte words to pinned host memory; each word is
// single-copy atomic on its own.
__device__ __forceinline__ void st_volatile_pair(unsigned long long* p, unsigned long long a,
                                                 unsigned long long b) {
    asm volatile("st.volatile.v2.u64 [%0], {%1, %2};" ::"l"(p), "l"(a), "l"(b) : "memory");
}

}  // namespace camelot
