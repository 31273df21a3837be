// Device entry points: the persistent pipeline kernel (all stage instances of
// a pipeline as CTA groups of one cooperative launch) and the direct launch of
// a single stage.
#include <cuda_runtime.h>

#include "pipeline_params.h"
#include "stage_dispatch.cuh"

namespace camelot {

// ---------------------------------------------------------------------------
// Leader side of the per-batch protocol (warp 0 of the instance's CTA 0).
// ---------------------------------------------------------------------------
struct LeaderState {
    unsigned long long seen_h;   // oldest waiting ticket the trigger has seen ...
    uint64_t seen_t;             // ... and since when (device clock)
    uint64_t idle_since;
    unsigned int polls;          // acquisition attempts (the host's stop flag is read on every 256th)
    unsigned int backoff_ns;     // stage 0, host queue: sleep between polls while nothing is published
};

__device__ __forceinline__ bool stop_requested(const PipeParams& P) {
    return *P.host_stop != 0ull || has_error(P.ctl);
}
// The stop flag lives in host memory: the acquisition loops read it on every
// 256th attempt only (well under a millisecond apart), and the device error
// word on every attempt.  Reads of host memory by idle leaders travel over the
// host link in the direction of the submits' copies: with dozens of instances
// polling, they cost the end-to-end path a quarter of its rate.
__device__ __forceinline__ bool stop_check(const PipeParams& P, LeaderState& ls) {
    return (ls.polls++ & 255u) == 0 ? stop_requested(P) : has_error(P.ctl);
}

// Claim a free slot of `r` for a new ticket (producer side).  Returns false on
// timeout (error recorded) or stop.
__device__ bool reserve_out(const PipeParams& P, const RingDev& r, uint32_t where,
                            unsigned long long* ticket) {
    Backoff bo(P.limit_ns);
    for (;;) {
        const unsigned long long t = *(volatile unsigned long long*)r.tail;
        const unsigned long long sq = ld_acquire_gpu(&r.seq[t % r.slots]);
        if (sq == t) {
            if (atomicCAS(r.tail, t, t + 1) == t) { *ticket = t; return true; }
            continue;
        }
        if (sq > t) continue;   // stale cursor
        if (stop_requested(P)) return false;
        if (!bo.step()) { record_error(P.ctl, DEV_ERR_OUT_SLOT, where); return false; }
    }
}

// Stage 0: the wait queue and batch trigger (Sec. 5.2 steps 1-2).  A batch of
// the oldest waiting tickets leaves when B of them are ready, or when the
// oldest has waited trig_wait_ns[k - 1] with k ready: max_wait_ns, or less when
// the QoS rule says that the wait plus the predicted latency of a k-query batch
// would pass QoS - margin.  Executed by warp 0 of the leader CTA; lane 0
// returns the command.  Records the arrival time and stream of the claimed
// tickets for the final stage.
__device__ unsigned int stage0_acquire(const PipeParams& P, LeaderState& ls,
                                       unsigned long long* first, unsigned int* n_out,
                                       bool* from_trace, long long* t_batch) {
    const int lane = threadIdx.x & 31;
    for (;;) {
        // every decision below is taken on lane 0's view, so the warp stays converged
        const int stop = __shfl_sync(0xffffffffu, lane == 0 ? (int)stop_check(P, ls) : 0, 0);
        if (stop) return CMD_EXIT;
        const unsigned long long h =
            __shfl_sync(0xffffffffu, *(volatile unsigned long long*)&P.ctl->in_head.v, 0);
        const uint64_t now = __shfl_sync(0xffffffffu, gtime(), 0);
        const TraceDev* tr = P.trace;
        const unsigned int armed = __shfl_sync(0xffffffffu, *(volatile unsigned int*)&tr->armed, 0);
        const unsigned long long tb =
            __shfl_sync(0xffffffffu, *(volatile unsigned long long*)&tr->base, 0);
        const unsigned long long tn =
            __shfl_sync(0xffffffffu, *(volatile unsigned long long*)&tr->n, 0);
        if (P.exit_after_trace && armed && h >= tb + tn) return CMD_EXIT;   // trace taken
        bool trace = armed && h >= tb && h < tb + tn;
        int avail;
        bool ready = false;
        long long arr = 0, oldest = 0;
        unsigned int sid = 0;
        if (trace) {
            unsigned long long t0 = 0;
            if (lane == 0) {
                t0 = *(volatile unsigned long long*)&P.ctl->trace_t0.v;
                if (t0 == 0ull) {
                    const unsigned long long prev = atomicCAS(&P.ctl->trace_t0.v, 0ull, now);
                    t0 = prev == 0ull ? now : prev;
                }
            }
            t0 = __shfl_sync(0xffffffffu, t0, 0);
            avail = (int)min((unsigned long long)P.B, tb + tn - h);
            if (lane < avail) {
                arr = (long long)t0 + tr->off[h - tb + lane];
                ready = (uint64_t)arr <= now;
            }
            oldest = (long long)t0 + tr->off[h - tb];
            sid = tr->stream_id;
        } else {
            // descriptors live in host memory: while the next one is not
            // published, one lane polls it alone (a read per poll instead of
            // B, which would take host-link bandwidth from the submits' copies)
            avail = P.B;
            const int first_ready = __shfl_sync(
                0xffffffffu, lane == 0 ? (int)(ld_acquire_sys(&P.qring[h & P.qmask].seq) == h + 1) : 0, 0);
            if (first_ready && lane < avail) {
                const QDesc& d = P.qring[(h + lane) & P.qmask];
                ready = ld_acquire_sys(&d.seq) == h + lane + 1;
                if (ready) { arr = d.t_arrival; sid = d.stream_id; }
            }
        }
        const unsigned int bal = __ballot_sync(0xffffffffu, ready);
        const int k = __ffs(~bal) - 1 < 0 ? 32 : __ffs(~bal) - 1;   // ready prefix length
        const int kk = min(k, avail);
        if (kk == 0) {
            const int idle_out = __shfl_sync(
                0xffffffffu, (!trace && now - ls.idle_since > (uint64_t)P.idle_ns) ? 1 : 0, 0);
            if (idle_out) return CMD_EXIT;
            if (trace) {
                __nanosleep(200);
            } else {
                // host queue empty: poll less and less often (0.5 .. 8 us)
                __nanosleep(ls.backoff_ns);
                ls.backoff_ns = min(2u * ls.backoff_ns, 8000u);
            }
            continue;
        }
        ls.backoff_ns = 500u;
        if (!trace && ls.seen_h != h) { ls.seen_h = h; ls.seen_t = now; }
        const uint64_t waited = trace ? (now - (uint64_t)oldest) : (now - ls.seen_t);
        if (kk < P.B && waited < (uint64_t)P.trig_wait_ns[kk - 1]) {
            __nanosleep(trace ? 200 : 1000);   // (host descriptors: fewer re-reads over the link)
            continue;
        }
        unsigned long long got = 0;
        if (lane == 0) got = atomicCAS(&P.ctl->in_head.v, h, h + kk);
        got = __shfl_sync(0xffffffffu, got, 0);
        if (got != h) continue;
        // the tickets [h, h + kk) are ours: record their metadata
        if (lane < kk) {
            QMeta& m = P.meta[(h + lane) & P.cmask];
            m.t_arrival = arr;
            m.stream_id = sid;
        }
        *first = h;
        *n_out = (unsigned)kk;
        *from_trace = trace;
        *t_batch = (long long)now;
        ls.idle_since = now;
        return CMD_WORK;
    }
}

// Stage s >= 1: take the oldest published batch of the input ring.
__device__ unsigned int stageN_acquire(const PipeParams& P, int s, LeaderState& ls,
                                       unsigned long long* slot_ticket, unsigned long long* first,
                                       unsigned int* n_out, long long* t_batch) {
    const RingDev& r = P.in_ring[s];
    const unsigned long long* up_tail = P.out_ring[s - 1].tail;
    const uint64_t bound = (uint64_t)P.idle_ns * (uint64_t)(s + 2) + (uint64_t)P.limit_ns;
    for (;;) {
        if (stop_check(P, ls)) return CMD_EXIT;
        const unsigned long long h = *(volatile unsigned long long*)r.head;
        const unsigned long long sq = ld_acquire_gpu(&r.seq[h % r.slots]);
        if (sq == h + 1) {
            if (atomicCAS(r.head, h, h + 1) != h) continue;
            const volatile BatchHdr* vh = &r.hdr[h % r.slots];
            const unsigned int hn = vh->n;
            if (hn == 0 || hn > (unsigned)P.B) {
                record_error(P.ctl, DEV_ERR_BAD_BATCH, s);
                return CMD_EXIT;
            }
            *slot_ticket = h;
            *first = vh->first;
            *n_out = hn;
            *t_batch = vh->t_batch;
            ls.idle_since = gtime();
            return CMD_WORK;
        }
        // empty: done once the upstream stage has exited and everything it
        // produced has been taken
        const unsigned long long ex = *(volatile unsigned long long*)&P.ctl->exited[s - 1].v;
        if (ex >= (unsigned long long)P.inst[s - 1] &&
            h >= *(volatile unsigned long long*)up_tail)
            return CMD_EXIT;
        if (gtime() - ls.idle_since > bound) {
            record_error(P.ctl, DEV_ERR_MAILBOX, 100 + s);
            return CMD_EXIT;
        }
        __nanosleep(300);
    }
}

template <uint32_t KINDS>
__global__ void __launch_bounds__(kThreads, 1) pipeline_kernel(const PipeParams* __restrict__ pp) {
    extern __shared__ float4 smem4[];
    const PipeParams& P = *pp;
    const int b = blockIdx.x;
    int s = 0;
    while (s + 1 < P.n_stages && b >= P.cta_begin[s + 1]) ++s;
    const int local = b - P.cta_begin[s];
    const int inst = local / P.quota[s];
    const int rank = local - inst * P.quota[s];
    GroupSync* gs = P.groups + P.inst_begin[s] + inst;
    StageCtx cx{rank, P.quota[s], gs, P.ctl, (uint64_t)P.limit_ns, (uint32_t)s,
                P.scratch + P.scratch_off[s] + (size_t)inst * P.inst_scratch[s],
                reinterpret_cast<float*>(smem4)};
    const StageParams& SP = P.st[s];
    const bool final_stage = (s == P.n_stages - 1);
    cx.defer_topk = final_stage;
    const bool leader = (rank == 0);

    __shared__ unsigned int sh_cmd, sh_n, sh_trace, sh_ok;
    __shared__ unsigned long long sh_in, sh_first, sh_out;
    __shared__ long long sh_tb;
    __shared__ unsigned long long sh_t_work;   // leader: when this batch's work was held
    LeaderState ls{~0ull, 0, gtime(), 0u, 500u};
    const bool tensor_stage = is_tensor_kind(SP.kind);
    if (tensor_stage) gemm_setup(reinterpret_cast<float*>(smem4));
    else if (SP.kind == KIND_NORM_POOL2_BF16) pool_setup(reinterpret_cast<float*>(smem4));
    else if (SP.kind == KIND_STREAM_SYNTH) stream_setup(reinterpret_cast<float*>(smem4));
    else if (SP.kind == KIND_MLP_FP32) mlp_setup(reinterpret_cast<float*>(smem4));
    const bool grouped = cx.nctas > 1;
    // the other CTAs wait for the leader's post for as long as the leader may idle
    const uint64_t post_wait = (uint64_t)P.idle_ns * (uint64_t)(P.n_stages + 2) + 2ull * (uint64_t)P.limit_ns;

    // Per batch: the leader acquires the work and posts it in the instance's
    // mailbox (releasing mb_gen = k + 1); every other CTA waits for that post,
    // runs its part of the body and adds one to the done count; the leader,
    // after its own part, waits for done = (k + 1) (CTAs - 1) and publishes the
    // batch.  One post and one count per batch, instead of two full barriers.
    for (unsigned int k = 0;; ++k) {
        // ---- the leader finds work and posts it
        if (leader) {
            if (threadIdx.x < 32) {
                unsigned int cmd, n = 0;
                unsigned long long in_t = 0, first = 0, out_t = 0;
                bool tr = false;
                long long tb = 0;
                const uint64_t t_acq = gtime();
                if (s == 0) {
                    cmd = stage0_acquire(P, ls, &first, &n, &tr, &tb);
                    in_t = first;
                } else {
                    if (threadIdx.x == 0) cmd = stageN_acquire(P, s, ls, &in_t, &first, &n, &tb);
                    cmd = __shfl_sync(0xffffffffu, cmd, 0);
                }
                if (threadIdx.x == 0) {
                    if (cmd == CMD_WORK) atomicAdd(&P.ctl->acq_ns[s].v, (unsigned long long)(gtime() - t_acq));
                    if (cmd == CMD_WORK && !final_stage && !reserve_out(P, P.out_ring[s], s, &out_t))
                        cmd = CMD_EXIT;
                    sh_t_work = gtime();
                    sh_cmd = cmd;
                    sh_n = n;
                    sh_in = in_t;
                    sh_out = out_t;
                    sh_tb = tb;
                    sh_trace = tr ? 1u : 0u;
                    sh_first = first;
                    if (grouped) {
                        gs->cmd = cmd;
                        gs->n = n;
                        gs->in_ticket = in_t;
                        gs->out_ticket = out_t;
                        gs->t_batch = tb;
                        gs->from_trace = tr ? 1u : 0u;
                        gs->first = first;
                        st_release_gpu32(&gs->mb_gen, k + 1u);
                    }
                }
            }
        } else if (threadIdx.x == 0) {
            if (wait_eq32(&gs->mb_gen, k + 1u, P.ctl, post_wait, 200 + s, DEV_ERR_MAILBOX)) {
                volatile GroupSync* vg = gs;
                sh_cmd = vg->cmd;
                sh_n = vg->n;
                sh_in = vg->in_ticket;
                sh_out = vg->out_ticket;
                sh_tb = vg->t_batch;
                sh_trace = vg->from_trace;
                sh_first = vg->first;
            } else {
                sh_cmd = CMD_EXIT;
            }
        }
        __syncthreads();
        if (sh_cmd != CMD_WORK) break;
        const int n = (int)sh_n;
        const unsigned long long first = sh_first;

        // ---- inputs and outputs of this batch
        RowRef in;
        if (s == 0) {
            if (sh_trace) {
                const TraceDev* tr = P.trace;
                in = RowRef{const_cast<char*>(tr->data) + (first - tr->base) * P.q_row, 0, ~0ull,
                            P.q_row};
            } else {
                in = RowRef{P.qdata, first, P.dmask, P.q_row};
            }
        } else {
            const RingDev& r = P.in_ring[s];
            in = RowRef{r.data + (sh_in % r.slots) * r.slot_bytes, 0, ~0ull, SP.in_row_bytes};
        }
        RowRef out{nullptr, 0, ~0ull, 0};
        if (!final_stage) {
            const RingDev& r = P.out_ring[s];
            out = RowRef{r.data + (sh_out % r.slots) * r.slot_bytes, 0, ~0ull, SP.out_row_bytes};
        }
        FinalOut fo{reinterpret_cast<int32_t*>(cx.scratch + SP.res_off),
                    reinterpret_cast<float*>(cx.scratch + SP.res_off) + (size_t)P.B * kMaxTopK,
                    RowRef{reinterpret_cast<char*>(P.sink), first, P.cmask, P.sink_ld * sizeof(float)}};
        if (P.sink == nullptr) fo.logits.base = nullptr;

        const uint64_t t_body = leader && threadIdx.x == 0 ? gtime() : 0;
        if (!stage_body<KINDS>(cx, SP, in, n, out, fo)) break;
        if (leader && threadIdx.x == 0) atomicAdd(&P.ctl->body_ns[s].v, (unsigned long long)(gtime() - t_body));

        // ---- end of the batch: the other CTAs report, the leader collects
        __syncthreads();
        if (!leader) {
            if (threadIdx.x == 0) {
                __threadfence();
                atomicAdd(&gs->done, 1u);
            }
            continue;
        }
        if (threadIdx.x == 0) {
            sh_ok = grouped ? wait_eq32(&gs->done, (k + 1u) * (unsigned)(cx.nctas - 1), P.ctl, P.limit_ns, 300 + s,
                                        DEV_ERR_GROUP_BARRIER)
                            : !has_error(P.ctl);
            __threadfence();
        }
        __syncthreads();
        if (!sh_ok) break;

        // ---- the leader publishes the result and releases the input
        if (final_stage && cx.defer_topk && tensor_stage && gemm_topk_cands(SP, n, cx.nctas)) {
            // the top-k candidates of every CTA are in (their done counts ordered them)
            gemm_cand_merge(cx, SP, n, fo, 0, kWarps);
            __syncthreads();
        }
        if (final_stage) {
            // completion records: data and flag in every 8-byte word (no
            // system-scope fence); the logits rows are ordered before them
            __shared__ long long sh_done;
            if (threadIdx.x == 0) sh_done = (long long)gtime();
            __syncthreads();
            if (P.sink != nullptr) __threadfence();
            const int kr = SP.res_k;
            for (int q = threadIdx.x; q < n; q += kThreads) {
                const unsigned long long t = first + q;
                const unsigned long long f = (unsigned long long)(uint32_t)(t + 1ull) << 32;
                const QMeta m = P.meta[t & P.cmask];
                uint32_t d[kCompWords];
                d[CW_STREAM] = m.stream_id;
                d[CW_STATUS] = 0u;
                d[CW_BATCH] = (uint32_t)n;
                d[CW_T_ARR] = (uint32_t)(unsigned long long)m.t_arrival;
                d[CW_T_ARR_HI] = (uint32_t)((unsigned long long)m.t_arrival >> 32);
                d[CW_T_BATCH] = (uint32_t)(unsigned long long)sh_tb;
                d[CW_T_BATCH_HI] = (uint32_t)((unsigned long long)sh_tb >> 32);
                d[CW_T_DONE] = (uint32_t)(unsigned long long)sh_done;
                d[CW_T_DONE_HI] = (uint32_t)((unsigned long long)sh_done >> 32);
#pragma unroll
                for (int r = 0; r < kMaxTopK; ++r) {
                    d[CW_IDX + r] = r < kr ? (uint32_t)fo.idx[(size_t)q * kr + r] : 0xffffffffu;
                    d[CW_VAL + r] = r < kr ? __float_as_uint(fo.val[(size_t)q * kr + r]) : 0u;
                }
#pragma unroll
                for (int i = CW_USED; i < kCompWords; ++i) d[i] = 0u;
                unsigned long long* w = P.comp[t & P.cmask].w;
#pragma unroll
                for (int i = 0; i < kCompWords; i += 2) st_volatile_pair(w + i, f | d[i], f | d[i + 1]);
            }
        } else if (threadIdx.x == 0) {
            const RingDev& r = P.out_ring[s];
            const unsigned int slot = (unsigned int)(sh_out % r.slots);
            BatchHdr& hd = r.hdr[slot];
            hd.first = first;
            hd.n = (unsigned)n;
            hd.t_batch = sh_tb;
            __threadfence();
            st_release_gpu(&r.seq[slot], sh_out + 1);
            if (r.note_pub != nullptr) {
                r.note_n[slot] = (unsigned)n;
                __threadfence_system();
                st_release_sys(&r.note_pub[slot], sh_out + 1);
            }
        }
        if (s == 0) {
            if (!sh_trace) {
                const unsigned long long R = P.qmask + 1;
                for (int q = threadIdx.x; q < n; q += kThreads)
                    st_release_sys(&P.qring[(first + q) & P.qmask].seq, first + q + R);
            }
        } else if (threadIdx.x == 0) {
            const RingDev& r = P.in_ring[s];
            const unsigned int slot = (unsigned int)(sh_in % r.slots);
            st_release_gpu(&r.seq[slot], sh_in + r.slots);
            if (r.note_free != nullptr) st_release_sys(&r.note_free[slot], sh_in + r.slots);
        }
        if (threadIdx.x == 0) {
            atomicAdd(&P.ctl->batches[s].v, 1ull);
            atomicAdd(&P.ctl->busy_ns[s].v, (unsigned long long)(gtime() - sh_t_work));
        }
        __syncthreads();   // the leader's shared mailbox copy is rewritten next
    }
    __syncthreads();
    if (tensor_stage) gemm_teardown(reinterpret_cast<float*>(smem4));
    if (leader && threadIdx.x == 0) {
        __threadfence();
        atomicAdd(&P.ctl->exited[s].v, 1ull);
        const unsigned long long st = ld_relaxed_gpu(&P.ctl->status.v);
        if (st != 0ull) *P.host_status = st;
    }
}

// Direct launch of one stage over one batch: the whole grid is one instance.
template <uint32_t KINDS>
__global__ void __launch_bounds__(kThreads, 1)
    stage_direct_kernel(const StageParams* __restrict__ sp, RowRef in, int n, RowRef out,
                        int32_t* idx, float* val, RowRef logits, char* scratch, GroupSync* gs,
                        Ctl* ctl, long long limit_ns) {
    extern __shared__ float4 smem4[];
    StageCtx cx{(int)blockIdx.x, (int)gridDim.x, gs, ctl, (uint64_t)limit_ns, 0u, scratch,
                reinterpret_cast<float*>(smem4)};
    FinalOut fo{idx, val, logits};
    const bool tensor_stage = is_tensor_kind(sp->kind);
    if (tensor_stage) gemm_setup(reinterpret_cast<float*>(smem4));
    else if (sp->kind == KIND_NORM_POOL2_BF16) pool_setup(reinterpret_cast<float*>(smem4));
    else if (sp->kind == KIND_STREAM_SYNTH) stream_setup(reinterpret_cast<float*>(smem4));
    else if (sp->kind == KIND_MLP_FP32) mlp_setup(reinterpret_cast<float*>(smem4));
    stage_body<KINDS>(cx, *sp, in, n, out, fo);
    if (tensor_stage) gemm_teardown(reinterpret_cast<float*>(smem4));
}

}  // namespace camelot

// Host-callable launch helpers (used by the runtime in runtime.cpp).
namespace camelot {

// The instantiations: the pipeline shapes of the workloads (the artifact
// kinds together), every other kind on its own (direct launches), and all
// kinds together (any other pipeline).
constexpr uint32_t kKindSets[] = {
    kind_bit(KIND_NORMALIZE_U8), kind_bit(KIND_NORM_POOL2_BF16), kind_bit(KIND_MLP_FP32),
    kind_bit(KIND_GEMM_BF16) | kind_bit(KIND_GEMM_FP8), kind_bit(KIND_NORMALIZE_U8_E4M3),
    kind_bit(KIND_EMBED_GATHER),
    kind_bit(KIND_NORMALIZE_U8) | kind_bit(KIND_MLP_FP32),
    kind_bit(KIND_NORM_POOL2_BF16) | kind_bit(KIND_GEMM_BF16) | kind_bit(KIND_GEMM_FP8),
    kind_bit(KIND_NORMALIZE_U8_E4M3) | kind_bit(KIND_GEMM_BF16) | kind_bit(KIND_GEMM_FP8),
    kind_bit(KIND_EMBED_GATHER) | kind_bit(KIND_GEMM_BF16) | kind_bit(KIND_GEMM_FP8),
    kind_bit(KIND_COMPUTE_SYNTH) | kind_bit(KIND_STREAM_SYNTH),
    kAllKinds};
constexpr int kNumSets = sizeof(kKindSets) / sizeof(kKindSets[0]);

template <int... I>
struct SetTable {
    static const void* const pipe[sizeof...(I)];
    static const void* const direct[sizeof...(I)];
};
template <int... I>
const void* const SetTable<I...>::pipe[sizeof...(I)] = {(const void*)pipeline_kernel<kKindSets[I]>...};
template <int... I>
const void* const SetTable<I...>::direct[sizeof...(I)] = {(const void*)stage_direct_kernel<kKindSets[I]>...};
using Table = SetTable<0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11>;
static_assert(kNumSets == 12, "instantiation table");

// The first (narrowest) instantiation holding every kind in `kinds`.
static int pick(uint32_t kinds) {
    for (int i = 0; i < kNumSets; ++i)
        if ((kKindSets[i] & kinds) == kinds) return i;
    return kNumSets - 1;
}

cudaError_t launch_pipeline_kernel(const PipeParams* dparams, int grid, cudaStream_t stream, uint32_t kinds) {
    void* args[] = {(void*)&dparams};
    return cudaLaunchCooperativeKernel(Table::pipe[pick(kinds)], dim3(grid), dim3(kThreads), args, kSmemBytes,
                                       stream);
}

cudaError_t launch_stage_direct(const StageParams* dsp, int kind, RowRef in, int n, RowRef out, int32_t* idx,
                                float* val, RowRef logits, char* scratch, GroupSync* gs, Ctl* ctl,
                                long long limit_ns, int grid, cudaStream_t stream) {
    void* args[] = {(void*)&dsp, &in, &n, &out, &idx, &val, &logits, &scratch, &gs, &ctl, &limit_ns};
    return cudaLaunchCooperativeKernel(Table::direct[pick(kind_bit(kind))], dim3(grid), dim3(kThreads), args,
                                       kSmemBytes, stream);
}

cudaError_t configure_kernels() {
    for (int i = 0; i < kNumSets; ++i) {
        cudaError_t e = cudaFuncSetAttribute(Table::pipe[i], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)kSmemBytes);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(Table::direct[i], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kSmemBytes);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t max_coresident_ctas(int* per_sm) {
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, Table::pipe[kNumSets - 1], kThreads,
                                                         kSmemBytes);
}
}  // namespace camelot
