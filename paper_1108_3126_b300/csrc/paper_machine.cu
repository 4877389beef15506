// paper_machine.cu -- the GPU machine of Section 8 (Rathnayake & Thielecke,
// SOS 2011), kept as a prior-art comparison (RX_VARIANT_PAPER).
//
// As the paper describes it: the tree nodes are an array d (the heap pi,
// with cont wired); one GPU thread per node; two integer vectors c and n of
// the same size.  c[i] = t means node i is to be simulated in macro step t,
// c[i] = -t that it already was (a process consumed by its message, Sec 7);
// n[j] = t+1 schedules node j for the next macro step.  Every launch is one
// micro-iteration: each thread whose node is scheduled simulates it (the
// transitions of Fig 4.2 / the processes of Sec 7), scheduling other nodes in
// c (evolution) or their continuations in n (a character matched), and
// raises one of two flags.  The host relaunches while c-activations happen;
// then swaps c and n and increments t (the n-way synchronisation).  Null has
// its own slot (index nn).  A claim is an atomic compare-and-swap t -> -t so
// each node is simulated at most once per macro step.
#include <cstring>
#include <utility>

#include "kernels.cuh"

namespace rx {

namespace {

__device__ __forceinline__ void sched(int* v, int j, int val, int* flag) {
    int old = v[j];
    if (old != val && old != -val) {
        atomicCAS(&v[j], old, val);
        *flag = 1;
    }
}

__global__ void k_paper_micro(const int4* __restrict__ d, int nn, int* c, int* nvec, int t, const uint8_t* w,
                              int64_t pos, int64_t len, int* flags) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nn) return;
    if (atomicCAS(&c[i], t, -t) != t) return;
    int4 x = d[i];
    int kind = x.x & 0xff, byte = (x.x >> 8) & 0xff;
    int k = x.w < 0 ? nn : x.w;  // cont, null slot = nn
    switch (kind) {
    case RX_ALT:
        sched(c, x.y, t, &flags[0]);
        sched(c, x.z, t, &flags[0]);
        break;
    case RX_CAT:
        sched(c, x.y, t, &flags[0]);
        break;
    case RX_STAR:
        sched(c, x.y, t, &flags[0]);
        sched(c, k, t, &flags[0]);
        break;
    case RX_EPS:
        sched(c, k, t, &flags[0]);
        break;
    default:  // CHAR: synchronise on the input character
        if (pos < len && w[pos] == byte) sched(nvec, k, t + 1, &flags[1]);
        break;
    }
}

__global__ void k_paper_init(int* c, int* nvec, int nn, int root, int* flags) {
    for (int i = threadIdx.x; i <= nn; i += blockDim.x) {
        c[i] = 0;
        nvec[i] = 0;
    }
    if (threadIdx.x == 0) {
        flags[0] = flags[1] = 0;
    }
    __syncthreads();
    if (threadIdx.x == 0) c[root] = 1;
}

}  // namespace

// One string; host-driven micro-iterations exactly as Section 8 describes.
// `scratch` (device) holds c, n (nn+1 ints each) and the flags; `hflags` is
// pinned host memory (3 ints) for the read-backs.  flags[0]: an activation
// in c during the last launch (relaunch); flags[1]: some character node
// matched during this macro step (else the machine is stuck).
cudaError_t paper_match_one(const DevTables& t, const uint8_t* str, int64_t len, int* scratch, int* hflags,
                            uint8_t* out_host, cudaStream_t st) {
    const int nn = t.nn;
    int* a = scratch;
    int* b = scratch + (nn + 1);
    int* flags = scratch + 2 * (nn + 1);
    k_paper_init<<<1, 256, 0, st>>>(a, b, nn, t.proot, flags);
    prof_count(1);
    int step = 1;
    const int threads = 128, blocks = (nn + threads - 1) / threads;
    for (int64_t pos = 0;; pos++) {
        cudaError_t e = cudaMemsetAsync(flags + 1, 0, sizeof(int), st);
        if (e != cudaSuccess) return e;
        for (;;) {
            e = cudaMemsetAsync(flags, 0, sizeof(int), st);
            if (e != cudaSuccess) return e;
            k_paper_micro<<<blocks, threads, 0, st>>>(t.pnodes, nn, a, b, step, str, pos, len, flags);
            prof_count(1);
            e = cudaMemcpyAsync(hflags, flags, 2 * sizeof(int), cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) return e;
            if (!hflags[0]) break;
        }
        if (pos == len) {
            e = cudaMemcpyAsync(&hflags[2], a + nn, sizeof(int), cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) return e;
            *out_host = (hflags[2] == step) ? 1 : 0;
            return cudaSuccess;
        }
        if (!hflags[1]) {  // stuck: nothing waits for the next character
            *out_host = 0;
            return cudaSuccess;
        }
        std::swap(a, b);
        step++;
    }
}

}  // namespace rx
