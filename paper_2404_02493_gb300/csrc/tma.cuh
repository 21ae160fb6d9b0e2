// Tensor-memory-accelerator (TMA) tile copies and mbarriers (sm_90+ PTX,
// used on sm_103a).
//
// A tile kernel's operands are described by CUtensorMaps built at setup
// (one table per (instance, level), see MapId): one thread issues one bulk
// tensor copy per operand region into shared memory, out-of-grid parts are
// zero-filled by the hardware, and completion is tracked by an mbarrier
// with the expected byte count.  Two buffers alternate, so the copies of a
// block's next tile are in flight while the current one is computed.
//
// Every wait is bounded (wall clock, TMA_WAIT_NS): on expiry the block
// records an error in the handle's error word, drains its copies (again
// bounded) and all of its threads leave together; the host reports
// MG_ETIMEOUT.
#pragma once
#include <stdint.h>

#include "common.cuh"

namespace wadr {

constexpr unsigned long long TMA_WAIT_NS = 100ull * 1000ull * 1000ull;   // 100 ms

__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* b, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* b, unsigned phase) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(b)), "r"(phase)
        : "memory");
    return ok != 0;
}
// Bounded wait for the completion of `phase`; false on expiry.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, unsigned phase) {
    if (mbar_try_wait(b, phase)) return true;
    const unsigned long long t0 = globaltimer_ns();
    while (!mbar_try_wait(b, phase)) {
        if (globaltimer_ns() - t0 > TMA_WAIT_NS) return false;
        __nanosleep(64);
    }
    return true;
}

// 2D / 3D tiled loads; x is the innermost coordinate (elements of the map's
// data type), must be 16-byte aligned in bytes.
__device__ __forceinline__ void tma_load_2d(void* dst, const void* map, int x, int y, uint64_t* b) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"(map), "r"(x), "r"(y), "r"(smem_u32(b))
        : "memory");
}
__device__ __forceinline__ void tma_load_3d(void* dst, const void* map, int x, int y, int z, uint64_t* b) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
            smem_u32(dst)),
        "l"(map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(b))
        : "memory");
}

// 1D bulk copy of `bytes` contiguous bytes (16-byte aligned addresses, size a
// multiple of 16).
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, uint64_t* b) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(b))
                 : "memory");
}

// Operand kinds of the tile kernels.  Complex slot maps are 3D over
// (2n reals, n rows, slots) of the level's slot allocation; quad maps are 3D
// over (4 components, n, n); real maps (k, sponge term) are 2D over (n, n).
// Box: (W, H) nodes; the kernels load each box at a node column that keeps
// the innermost byte offset a multiple of 16.
enum MapId : int {
    MC_CHEB_X = 0,   // complex, (CTX+4) x (CTY+4)        from (x0-2, y0-2)
    MC_CHEB_G,       // complex, (CTX+4) x (CTY+2)        from (x0-2, y0-1)
    MC_CHEB_D,       // complex, CTX x CTY                from (x0, y0)
    MK_CHEB,         // k,       (CTX+8) x (CTY+2)        from (x0-4, y0-1)
    MS_CHEB,         // sponge,  same box
    MC_RESTR,        // complex, (RFW+3) x (RFH+2)        from (fx0-2, fy0-1)
    MK_RESTR,        // k,       (RFW+7) x (RFH+2)        from (fx0-4, fy0-1)
    MS_RESTR,
    MC_PROL_E,       // complex (coarse level), (PCW+1) x PCH  from (cx0-1, cy0)
    MC_PROL_X,       // complex, (PTX+4) x (PTY+2)        from (x0-2, y0-1)
    MC_PROL_T,       // complex, PTX x PTY                from (x0, y0)
    MQ_PROL,         // quads,   PTX x PTY
    MK_PROL,         // k,       PTX x PTY
    MS_PROL,
    MC_PRE_K2,                            // complex, (2CX+4) x (2CY+3)  from (fx0-2, fy0-1), per pre candidate
    MC_PRE_K01 = MC_PRE_K2 + 5,           // complex, (2CX+2) x (2CY+1)  from (fx0, fy0)
    MQ_PRE = MC_PRE_K01 + 5,              // quads,   (2CX+1) x (2CY+1)  from (fx0, fy0)
    NMAP = MQ_PRE + 5
};
constexpr int TMAP_BYTES = 128;   // sizeof(CUtensorMap)

__device__ __forceinline__ const void* tmap(const LevelDesc& d, int id) {
    return reinterpret_cast<const unsigned char*>(d.tm) + (size_t)id * TMAP_BYTES;
}

// Two-buffer TMA pipeline of a block: thread 0 initialises the barriers
// and issues the copies; every thread waits.  A failed wait sets the
// handle's error word, drains and makes every thread leave.
struct TmaPipe {
    uint64_t* bar;     // 2 mbarriers in shared memory
    unsigned phase[2];
    bool pending[2];   // buffer has copies in flight (thread 0's view)
    __device__ __forceinline__ void init(uint64_t* b2) {
        bar = b2;
        phase[0] = phase[1] = 0;
        pending[0] = pending[1] = false;
        if (threadIdx.x == 0 && threadIdx.y == 0) {
            mbar_init(&bar[0], 1);
            mbar_init(&bar[1], 1);
            fence_mbar_init();
        }
        __syncthreads();
    }
    // thread 0, before issuing the copies of buffer b
    __device__ __forceinline__ void expect(int b, unsigned bytes) {
        mbar_expect_tx(&bar[b], bytes);
        pending[b] = true;
    }
    // true if buffer b's copies landed (block-uniform).  On expiry: error
    // word set, false for every thread, after thread 0 has waited once more
    // (bounded) for the copies still in flight into this block's shared
    // memory: those of buffer b and, if issued, of the other buffer.  The
    // copies read device memory and complete within microseconds unless the
    // memory system has failed; if even the second limit passes, the context
    // is lost anyway and the block leaves without them.
    __device__ __forceinline__ bool wait(int b, unsigned* err) {
        const bool ok = __syncthreads_and(mbar_wait(&bar[b], phase[b]) ? 1 : 0) != 0;
        phase[b] ^= 1;
        pending[b] = false;
        if (!ok) {
            if (threadIdx.x == 0 && threadIdx.y == 0) {
                if (err) atomicExch(err, 1u);
                mbar_wait(&bar[b], phase[b] ^ 1);
                if (pending[b ^ 1]) mbar_wait(&bar[b ^ 1], phase[b ^ 1]);
            }
            __syncthreads();
        }
        return ok;
    }
};

// Typed pieces of the dynamic shared memory, each 128-byte aligned (TMA
// destinations).  The first piece starts at the next 128-byte boundary of
// the dynamic block; sizes include that slack.
struct TmaCarve {
    uintptr_t p;
    __device__ __forceinline__ explicit TmaCarve(unsigned char* base)
        : p(((uintptr_t)base + 127) & ~(uintptr_t)127) {}
    template <typename E>
    __device__ __forceinline__ E* take(int count) {
        E* r = reinterpret_cast<E*>(p);
        p += ((uintptr_t)count * sizeof(E) + 127) & ~(uintptr_t)127;
        return r;
    }
};
template <typename E> __host__ __device__ constexpr int tma_piece(int count) {
    return (int)(((size_t)count * sizeof(E) + 127) / 128 * 128);
}

}  // namespace wadr
