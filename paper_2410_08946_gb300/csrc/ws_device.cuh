// ws_device.cuh -- device-side helpers shared by the libws kernels:
// image geometry, neighbourhood offsets, the device status word and a
// bounded device-wide barrier for cooperative (co-resident) launches.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ws {

// ---------------------------------------------------------------------------
// status word (one per context, in device memory)
// ---------------------------------------------------------------------------

enum : int {
    DEV_OK = 0,
    DEV_NONCONVERGED = 5,
    DEV_TIMEOUT = 6,
    DEV_EDGE_TABLE_FULL = 3,
    DEV_BAD_LABELS = 1,
};

struct DevStatus {
    int code;            // first error recorded (0 = none)
    int where;           // which loop recorded it
    int abort;           // set with any error: cooperative loops leave at once
    int pad0;
    unsigned bar_count;  // device-wide barrier: arrivals in the current phase
    unsigned bar_gen;    // device-wide barrier: generation counter
    int changed[4];      // per-round change counters (rotating)
    int rounds_plateau;  // rounds the step II relaxation took (diagnostics)
    int rounds_jump;     // rounds the step III pointer jumping took
    long long edges;     // distinct region pairs found by the adjacency pass
    int pad1[6];
};

__device__ __forceinline__ void record_error(DevStatus *s, int code, int where)
{
    if (atomicCAS(&s->code, 0, code) == 0) s->where = where;
    atomicExch(&s->abort, 1);
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Device-wide barrier for a cooperative launch (all blocks co-resident).
// Bounded: a block that waits longer than timeout_ns records DEV_TIMEOUT and
// every waiting block returns false (the caller then leaves the kernel).
// bar_count must be 0 when the kernel starts.  Bit 63 of timeout_ns (kHold,
// set only by failure-detection tests) makes block 0 return false without
// arriving, so that the other blocks' waits run out.
constexpr unsigned long long kHold = 1ull << 63;

__device__ __forceinline__ bool grid_barrier(DevStatus *s, unsigned long long timeout_ns)
{
    __shared__ int ok_s;
    __syncthreads();
    if ((timeout_ns & kHold) && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0) return false;
    timeout_ns &= ~kHold;
    if (threadIdx.x == 0) {
        int ok = 1;
        volatile unsigned *vgen = &s->bar_gen;
        volatile int *vabort = &s->abort;
        const unsigned nblocks = gridDim.x * gridDim.y * gridDim.z;
        unsigned gen = *vgen;
        __threadfence();
        unsigned arrived = atomicAdd(&s->bar_count, 1u);
        if (arrived == nblocks - 1) {
            atomicExch(&s->bar_count, 0u);
            __threadfence();
            atomicAdd(&s->bar_gen, 1u);
        } else {
            unsigned long long t0 = global_ns();
            while (*vgen == gen) {
                if (*vabort) {
                    ok = 0;
                    break;
                }
                if (global_ns() - t0 > timeout_ns) {
                    record_error(s, DEV_TIMEOUT, 100);
                    ok = 0;
                    break;
                }
                __nanosleep(40);
            }
        }
        __threadfence();
        ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
}

// ---------------------------------------------------------------------------
// geometry
// ---------------------------------------------------------------------------

struct Geo {
    int W, H, D;  // D == 1 for 2D images
    int HW;       // W * H
    int N;        // W * H * D (< 2^31)
};

// Neighbour offsets in ascending linear-index order (dz, then dy, then dx),
// which is the order Eq. 1's tie-break ("the largest index") refers to.
// A 2D pipeline may run on one of several tile shapes: the template value
// CONN + 100 * shape names connectivity CONN on tile shape `shape`
// (ws_tuning.tile_shape), with the neighbourhood of CONN % 100.
template <int CONN> struct Nb : Nb<CONN % 100> {};

template <> struct Nb<4> {
    static constexpr int n = 4;
    __device__ static constexpr int dx(int i) { return i == 1 ? -1 : (i == 2 ? 1 : 0); }
    __device__ static constexpr int dy(int i) { return i == 0 ? -1 : (i == 3 ? 1 : 0); }
    __device__ static constexpr int dz(int) { return 0; }
};

template <> struct Nb<8> {
    static constexpr int n = 8;
    // (dy, dx): (-1,-1) (-1,0) (-1,1) (0,-1) (0,1) (1,-1) (1,0) (1,1)
    __device__ static constexpr int dx(int i)
    {
        return (i == 0 || i == 3 || i == 5) ? -1 : ((i == 1 || i == 6) ? 0 : 1);
    }
    __device__ static constexpr int dy(int i) { return i < 3 ? -1 : (i < 5 ? 0 : 1); }
    __device__ static constexpr int dz(int) { return 0; }
};

template <> struct Nb<6> {
    static constexpr int n = 6;
    __device__ static constexpr int dx(int i) { return i == 2 ? -1 : (i == 3 ? 1 : 0); }
    __device__ static constexpr int dy(int i) { return i == 1 ? -1 : (i == 4 ? 1 : 0); }
    __device__ static constexpr int dz(int i) { return i == 0 ? -1 : (i == 5 ? 1 : 0); }
};

// 26-connectivity: every (dz, dy, dx) in {-1, 0, 1}^3 but the centre, in
// ascending linear-offset order (cell c = 9 (dz + 1) + 3 (dy + 1) + dx + 1,
// the centre c = 13 skipped)
template <> struct Nb<26> {
    static constexpr int n = 26;
    __device__ static constexpr int cell(int i) { return i < 13 ? i : i + 1; }
    __device__ static constexpr int dx(int i) { return cell(i) % 3 - 1; }
    __device__ static constexpr int dy(int i) { return (cell(i) / 3) % 3 - 1; }
    __device__ static constexpr int dz(int i) { return cell(i) / 9 - 1; }
};

template <int CONN> struct Dim {
    static constexpr int nd = (CONN % 100 == 4 || CONN % 100 == 8) ? 2 : 3;
};

// Forward half of the neighbourhood: offsets whose linear index delta is
// positive (indices n/2 .. n-1 of the ascending order).
template <int CONN> struct Half {
    static constexpr int first = Nb<CONN>::n / 2;
};

__device__ __forceinline__ int imin(int a, int b) { return a < b ? a : b; }
__device__ __forceinline__ int imax(int a, int b) { return a > b ? a : b; }

}  // namespace ws
