// Cross-process batch ring (Sec. 6.2: microservices in separate processes hand
// their global-memory outputs to the next stage through CUDA IPC handles).
// One device allocation of `slots` slots exported with cudaIpcGetMemHandle, and
// two inter-process events per slot (ready: the producer's writes are done;
// free: the consumer's reads are done).  All ordering on the GPU is by stream
// waits on those events, so no kernel of one process ever waits for a kernel of
// the other; the host sides sequence their calls over their own channel.
#include <cuda_runtime.h>

#include <cstring>

#include "../../include/camelot.h"

camelot_status camelot_internal_fail(camelot_status st, const char* msg);

static_assert(sizeof(cudaIpcMemHandle_t) <= 64, "IPC memory handle size");
static_assert(sizeof(cudaIpcEventHandle_t) <= 64, "IPC event handle size");

struct camelot_xring {
    bool producer = false;
    int device = 0;
    char* base = nullptr;
    uint64_t slot_bytes = 0, stride = 0;
    uint32_t slots = 0;
    cudaEvent_t ready[CAMELOT_XRING_MAX_SLOTS] = {};
    cudaEvent_t freed[CAMELOT_XRING_MAX_SLOTS] = {};
};

static void xring_free(camelot_xring* x) {
    if (!x) return;
    for (uint32_t k = 0; k < CAMELOT_XRING_MAX_SLOTS; ++k) {
        if (x->ready[k]) cudaEventDestroy(x->ready[k]);
        if (x->freed[k]) cudaEventDestroy(x->freed[k]);
    }
    if (x->base) {
        if (x->producer) cudaFree(x->base);
        else cudaIpcCloseMemHandle(x->base);
    }
    delete x;
}

static uint64_t slot_stride(uint64_t slot_bytes) { return (slot_bytes + 255) / 256 * 256; }

extern "C" camelot_status camelot_xring_create(uint64_t slot_bytes, uint32_t slots, camelot_xring** out,
                                               camelot_xring_handle* h) {
    if (!out || !h || slot_bytes == 0 || slots < 1 || slots > CAMELOT_XRING_MAX_SLOTS)
        return camelot_internal_fail(CAMELOT_EINVAL, "need slot_bytes > 0, 1..64 slots and output pointers");
    *out = nullptr;
    auto* x = new camelot_xring();
    x->producer = true;
    x->slot_bytes = slot_bytes;
    x->stride = slot_stride(slot_bytes);
    x->slots = slots;
    memset(h, 0, sizeof(*h));
    cudaError_t e = cudaGetDevice(&x->device);
    if (e == cudaSuccess) e = cudaMalloc((void**)&x->base, x->stride * slots);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        xring_free(x);
        return camelot_internal_fail(CAMELOT_ENOMEM, "ring allocation failed");
    }
    cudaIpcMemHandle_t mh;
    if (e == cudaSuccess) e = cudaIpcGetMemHandle(&mh, x->base);
    for (uint32_t k = 0; k < slots && e == cudaSuccess; ++k) {
        const unsigned flags = cudaEventDisableTiming | cudaEventInterprocess;
        cudaIpcEventHandle_t eh;
        e = cudaEventCreateWithFlags(&x->ready[k], flags);
        if (e == cudaSuccess) e = cudaIpcGetEventHandle(&eh, x->ready[k]);
        if (e == cudaSuccess) memcpy(h->ready[k], &eh, sizeof(eh));
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&x->freed[k], flags);
        if (e == cudaSuccess) e = cudaIpcGetEventHandle(&eh, x->freed[k]);
        if (e == cudaSuccess) memcpy(h->free_[k], &eh, sizeof(eh));
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        xring_free(x);
        return camelot_internal_fail(CAMELOT_ECUDA, "IPC ring creation failed");
    }
    h->slot_bytes = slot_bytes;
    h->slots = slots;
    h->device = x->device;
    memcpy(h->mem, &mh, sizeof(mh));
    *out = x;
    return CAMELOT_OK;
}

extern "C" camelot_status camelot_xring_open(const camelot_xring_handle* h, camelot_xring** out) {
    if (!h || !out || h->slot_bytes == 0 || h->slots < 1 || h->slots > CAMELOT_XRING_MAX_SLOTS)
        return camelot_internal_fail(CAMELOT_EINVAL, "malformed ring handle");
    *out = nullptr;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != h->device)
        return camelot_internal_fail(CAMELOT_EINVAL, "the ring lives on another device");
    auto* x = new camelot_xring();
    x->device = dev;
    x->slot_bytes = h->slot_bytes;
    x->stride = slot_stride(h->slot_bytes);
    x->slots = h->slots;
    cudaIpcMemHandle_t mh;
    memcpy(&mh, h->mem, sizeof(mh));
    cudaError_t e = cudaIpcOpenMemHandle((void**)&x->base, mh, cudaIpcMemLazyEnablePeerAccess);
    if (e != cudaSuccess) x->base = nullptr;
    for (uint32_t k = 0; k < x->slots && e == cudaSuccess; ++k) {
        cudaIpcEventHandle_t eh;
        memcpy(&eh, h->ready[k], sizeof(eh));
        e = cudaIpcOpenEventHandle(&x->ready[k], eh);
        if (e == cudaSuccess) {
            memcpy(&eh, h->free_[k], sizeof(eh));
            e = cudaIpcOpenEventHandle(&x->freed[k], eh);
        }
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        xring_free(x);
        return camelot_internal_fail(CAMELOT_ECUDA, "the ring handle does not open in this process");
    }
    *out = x;
    return CAMELOT_OK;
}

extern "C" void* camelot_xring_slot(const camelot_xring* x, uint32_t k) {
    if (!x || k >= x->slots) return nullptr;
    return x->base + (uint64_t)k * x->stride;
}

static camelot_status side_call(camelot_xring* x, uint32_t k, void* stream, bool want_producer, bool wait,
                                cudaEvent_t* evs) {
    if (!x || k >= x->slots) return camelot_internal_fail(CAMELOT_EINVAL, "bad ring or slot");
    if (x->producer != want_producer) return camelot_internal_fail(CAMELOT_EINVAL, "call made on the wrong side");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const cudaError_t e = wait ? cudaStreamWaitEvent(st, evs[k], 0) : cudaEventRecord(evs[k], st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return camelot_internal_fail(CAMELOT_ECUDA, wait ? "stream wait failed" : "event record failed");
    }
    return CAMELOT_OK;
}

extern "C" camelot_status camelot_xring_produce_begin(camelot_xring* x, uint32_t k, void* stream) {
    return side_call(x, k, stream, true, true, x ? x->freed : nullptr);
}
extern "C" camelot_status camelot_xring_produce_end(camelot_xring* x, uint32_t k, void* stream) {
    return side_call(x, k, stream, true, false, x ? x->ready : nullptr);
}
extern "C" camelot_status camelot_xring_consume_begin(camelot_xring* x, uint32_t k, void* stream) {
    return side_call(x, k, stream, false, true, x ? x->ready : nullptr);
}
extern "C" camelot_status camelot_xring_consume_end(camelot_xring* x, uint32_t k, void* stream) {
    return side_call(x, k, stream, false, false, x ? x->freed : nullptr);
}

extern "C" camelot_status camelot_xring_destroy(camelot_xring* x) {
    if (!x) return camelot_internal_fail(CAMELOT_EINVAL, "null ring");
    xring_free(x);
    return CAMELOT_OK;
}
