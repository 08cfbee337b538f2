// Create-time kernels: internal cell numbering and the slab layout of the
// netlist for the wirelength kernel (k_wire.cu).  All of them run once per
// handle; nothing here is on the per-iteration path.
//
// Cell numbering: cells whose index is a multiple of kSeedStride start as
// region seeds labelled with their own index; each round, a net (of at most
// kRankMaxDegree pins) takes the smallest label among its cells and every
// cell the smallest label among its nets (Jacobi rounds, so the result does
// not depend on the order in which threads run).  A cell keeps the round in
// which its label last dropped as its distance.  The host then numbers the
// cells by (label, distance, index): the cells of one region get consecutive
// numbers, and so do the pins of most nets.
#include "fftpl_internal.cuh"

namespace fftpl {

constexpr int kIntMax = 0x7fffffff;

__global__ void k_lp_init(int m, int stride, int* __restrict__ lab, int* __restrict__ dist) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    bool seed = (i % stride) == 0;
    lab[i] = seed ? i : kIntMax;
    dist[i] = seed ? 0 : kIntMax;
}

// netlab[e] = min label over the movable cells of net e (2 <= d <= maxd)
__global__ void k_lp_net(int E, const int* __restrict__ np, const int* __restrict__ pc, int m,
                         int maxd, const int* __restrict__ lab, int* __restrict__ netlab) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= E) return;
    int p0 = np[e], p1 = np[e + 1], v = kIntMax;
    if (p1 - p0 >= 2 && p1 - p0 <= maxd)
        for (int p = p0; p < p1; ++p) {
            int cc = pc[p];
            if (cc < m) v = min(v, lab[cc]);
        }
    netlab[e] = v;
}

// next[c] = min(next[c], netlab[e]) for every movable cell c of net e
__global__ void k_lp_cell(int E, const int* __restrict__ np, const int* __restrict__ pc, int m,
                          const int* __restrict__ netlab, int* __restrict__ next) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= E) return;
    int v = netlab[e];
    if (v == kIntMax) return;
    for (int p = np[e]; p < np[e + 1]; ++p) {
        int cc = pc[p];
        if (cc < m) atomicMin(next + cc, v);
    }
}

// lab <- next, distance = round + 1 where the label dropped
__global__ void k_lp_step(int m, int round, int* __restrict__ lab, const int* __restrict__ next,
                          int* __restrict__ dist) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    int a = lab[i], b = next[i];
    if (b < a) {
        lab[i] = b;
        dist[i] = round + 1;
    }
}

// key[e] = smallest internal number among the movable cells of net e (m if
// none)
__global__ void k_net_key(int E, const int* __restrict__ np, const int* __restrict__ pc, int m,
                          const int* __restrict__ rank, int* __restrict__ key) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= E) return;
    int v = m;
    for (int p = np[e]; p < np[e + 1]; ++p) {
        int cc = pc[p];
        if (cc < m) v = min(v, rank[cc]);
    }
    key[e] = v;
}

// Pin records in slab layout: pin k of net e at net_slot[e] + 32 k.  A pin
// on a movable cell stores its cell's internal number and its offset; a pin
// on a fixed cell stores -1 and its absolute coordinate fl32(centre +
// offset).  cslot (deterministic mode, else null): each pin's slot in the
// cell-ordered pin array.
__global__ void k_fill_slabs(int E, const int* __restrict__ np, const int* __restrict__ pc,
                             const float* __restrict__ dx, const float* __restrict__ dy, int m,
                             const int* __restrict__ rank, const float* __restrict__ fix_x,
                             const float* __restrict__ fix_y, const int* __restrict__ net_slot,
                             const int* __restrict__ net_lanes, const int* __restrict__ cslot,
                             int* __restrict__ spc, float* __restrict__ sdx,
                             float* __restrict__ sdy, int* __restrict__ sslot) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= E) return;
    const int base = net_slot[e];
    if (base < 0) return;
    // L lanes per net: pin k at base + 32 (k / L) + k % L (L = 1: base + 32 k)
    const int L = net_lanes[e];
    const int p0 = np[e], d = np[e + 1] - p0;
    for (int k = 0; k < d; ++k) {
        const int p = p0 + k;
        const size_t slot = (size_t)base + 32 * (size_t)(k / L) + (size_t)(k % L);
        const int cc = pc[p];
        if (cc < m) {
            spc[slot] = rank[cc];
            sdx[slot] = dx[p];
            sdy[slot] = dy[p];
        } else {
            spc[slot] = -1;
            sdx[slot] = __fadd_rn(fix_x[cc - m], dx[p]);
            sdy[slot] = __fadd_rn(fix_y[cc - m], dy[p]);
        }
        if (sslot) sslot[slot] = cslot[p];
    }
}

static inline unsigned nb(long long n) { return (unsigned)((n + 255) / 256); }

cudaError_t launch_label_rounds(int m, int E, const int* np, const int* pc, int* lab, int* next,
                                int* dist, int* netlab, cudaStream_t s) {
    if (m <= 0) return cudaSuccess;
    k_lp_init<<<nb(m), 256, 0, s>>>(m, kSeedStride, lab, dist);
    // no nets: every cell keeps its seed label (or none) at distance 0 / unset
    for (int r = 0; r < (E > 0 ? kLabelRounds : 0); ++r) {
        k_lp_net<<<nb(E), 256, 0, s>>>(E, np, pc, m, kRankMaxDegree, lab, netlab);
        cudaError_t e = cudaMemcpyAsync(next, lab, (size_t)m * sizeof(int), cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return e;
        k_lp_cell<<<nb(E), 256, 0, s>>>(E, np, pc, m, netlab, next);
        k_lp_step<<<nb(m), 256, 0, s>>>(m, r, lab, next, dist);
    }
    return cudaGetLastError();
}

cudaError_t launch_net_key(int m, int E, const int* np, const int* pc, const int* rank, int* key,
                           cudaStream_t s) {
    if (E <= 0) return cudaSuccess;
    k_net_key<<<nb(E), 256, 0, s>>>(E, np, pc, m, rank, key);
    return cudaGetLastError();
}

cudaError_t launch_fill_slabs(int m, int E, const int* np, const int* pc, const float* dx,
                              const float* dy, const int* rank, const float* fix_x,
                              const float* fix_y, const int* net_slot, const int* net_lanes,
                              const int* cslot, int* spc, float* sdx, float* sdy, int* sslot,
                              cudaStream_t s) {
    if (E <= 0) return cudaSuccess;
    k_fill_slabs<<<nb(E), 256, 0, s>>>(E, np, pc, dx, dy, m, rank, fix_x, fix_y, net_slot,
                                       net_lanes, cslot, spc, sdx, sdy, sslot);
    return cudaGetLastError();
}

}  // namespace fftpl
