// hrm_common.cuh -- device helpers shared by the libhrm CUDA kernels.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace hrm {

// Kernel-side error codes written to the workspace error word (first writer wins).
enum DeviceError : unsigned {
    DEV_OK = 0,
    DEV_SLOT_OVERFLOW = 1,   // internal: slot table could not make progress
    DEV_BAD_JOB = 2,         // batch: malformed job descriptor
    DEV_QUEUE_TIMEOUT = 3,   // bounded spin on a queue/flag gave up
};

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// Per-half unsigned 16-bit min/max of packed pairs (native on sm_90+).
__device__ __forceinline__ uint32_t vmin2(uint32_t a, uint32_t b) {
    uint32_t d;
    asm("min.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}
__device__ __forceinline__ uint32_t vmax2(uint32_t a, uint32_t b) {
    uint32_t d;
    asm("max.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}

// byte permute: result byte i = byte[(s >> 4i) & 7] of {b:a} (a = bytes 0..3).
__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t s) {
    return __byte_perm(a, b, s);
}

// Unpack four 8-bit counts c0..c3 of `w` into two 16-bit pairs (c0|c1<<16), (c2|c3<<16).
__device__ __forceinline__ uint32_t lo_pair(uint32_t w) { return __byte_perm(w, 0u, 0x4140); }
__device__ __forceinline__ uint32_t hi_pair(uint32_t w) { return __byte_perm(w, 0u, 0x4342); }

__device__ __forceinline__ int bitlen(uint32_t x) { return x ? 32 - __clz(x) : 0; }

template <typename T>
__device__ __forceinline__ uint32_t ldpx(const unsigned char* base, size_t pitch, int x, int y) {
    return (uint32_t)__ldg(reinterpret_cast<const T*>(base + (size_t)y * pitch) + x);
}

__device__ __forceinline__ void set_error(unsigned* err, unsigned code) {
    if (err) atomicCAS(err, 0u, code);
}

}  // namespace hrm
