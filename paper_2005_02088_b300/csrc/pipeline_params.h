// Plain-data layout of a pipeline's rings and of the persistent kernel's
// parameters, shared by the host runtime and the device code.
#pragma once
#include <cstddef>
#include <cstdint>

#include "../../include/camelot.h"
#include "device_sync.cuh"
#include "stage_params.h"

namespace camelot {

// Header of one inter-stage batch slot.  A batch is a run of consecutive query
// tickets [first, first + n).
struct BatchHdr {
    unsigned long long first;
    unsigned int n;
    unsigned int pad;
    long long t_batch;
    long long pad2;
};

// Device view of one batch ring (Vyukov bounded queue): slot i starts with
// seq = i ("empty for ticket i"); the producer of ticket t waits for seq == t,
// fills the slot and releases seq = t + 1; the consumer of ticket t waits for
// seq == t + 1, reads the slot in place and releases seq = t + slots.
struct RingDev {
    unsigned long long* seq;       // device [slots]
    BatchHdr* hdr;                 // device [slots]
    char* data;                    // device [slots][slot_bytes]
    unsigned long long* head;      // device: consumer cursor
    unsigned long long* tail;      // device: producer cursor
    unsigned int slots;
    unsigned int pad;
    size_t slot_bytes;
    // host-staged handoff only (pinned, mapped host memory; else null):
    volatile unsigned long long* note_pub;   // producer side: t + 1 once ticket t is published
    volatile unsigned int* note_n;           // producer side: rows of ticket t's batch
    volatile unsigned long long* note_free;  // consumer side: t + slots once ticket t is released
};

// Host query ring entry (pinned, mapped host memory).  Same protocol as the
// batch rings with one query per ticket; the query bytes are in the parallel
// data array.
struct QDesc {
    volatile unsigned long long seq;
    long long t_arrival;
    unsigned int stream_id;
    unsigned int pad;
    unsigned long long pad2;
};

// Completion ring entry (pinned, mapped host memory), indexed by ticket t.
// Every 8-byte word carries 32 bits of the completion in its low half and the
// flag (t + 1, truncated to 32 bits) in its high half.  Aligned 8-byte stores
// are single-copy atomic, so the host holds a whole record once every word
// shows the flag: the device writes data and flags together, with no
// system-scope fence between them.
enum CompWord : int {
    CW_STREAM = 0, CW_STATUS, CW_BATCH, CW_T_ARR, CW_T_ARR_HI, CW_T_BATCH, CW_T_BATCH_HI, CW_T_DONE,
    CW_T_DONE_HI, CW_IDX, CW_VAL = CW_IDX + kMaxTopK, CW_USED = CW_VAL + kMaxTopK
};
constexpr int kCompWords = (CW_USED + 1) / 2 * 2;   // whole 16-byte pairs
struct alignas(16) CompSlot {
    unsigned long long w[kCompWords];
};

// Per-query metadata the batch trigger records for the final stage (device
// memory, indexed by ticket like the completion ring).
struct QMeta {
    long long t_arrival;
    unsigned int stream_id;
    unsigned int pad;
};

// A trace of device-resident queries (device memory).
struct TraceDev {
    const char* data;          // query rows
    const long long* off;      // arrival offsets, ns
    unsigned long long base;   // first ticket
    unsigned long long n;
    unsigned int stream_id;
    unsigned int armed;
};

enum Cmd : unsigned int { CMD_NONE = 0, CMD_WORK = 1, CMD_EXIT = 2 };

struct PipeParams {
    int n_stages;
    int B;                      // batch size of the trigger
    int handoff;                // camelot_handoff
    int total_ctas;
    int cta_begin[kMaxStages + 1];
    int inst[kMaxStages];
    int quota[kMaxStages];
    int inst_begin[kMaxStages];
    size_t inst_scratch[kMaxStages];   // scratch bytes per instance of stage s
    size_t scratch_off[kMaxStages];    // offset of stage s's first instance
    StageParams st[kMaxStages];
    RingDev out_ring[kMaxStages];      // producer view of stage s's output (s < n-1)
    RingDev in_ring[kMaxStages];       // consumer view of stage s's input (s >= 1)
    Ctl* ctl;
    volatile unsigned long long* host_stop;     // pinned: host sets to 1 to stop
    volatile unsigned long long* host_status;   // pinned: device mirrors its first error
    GroupSync* groups;
    char* scratch;
    QDesc* qring;
    char* qdata;
    unsigned long long qmask;       // query descriptor ring (= completion ring) mask
    unsigned long long dmask;       // query data ring mask
    size_t q_row;
    CompSlot* comp;
    QMeta* meta;                // device [cmask + 1]
    unsigned long long cmask;
    float* sink;
    size_t sink_ld;             // floats per sink row
    TraceDev* trace;
    long long max_wait_ns, idle_ns, limit_ns;
    int exit_after_trace;
    // batch trigger: a batch of b < B ready queries leaves once its oldest has
    // waited trig_wait_ns[b - 1] (max_wait_ns, or less under the QoS rule)
    long long trig_wait_ns[32];
};

}  // namespace camelot
