// Coarse-grained collision detection on the Eulerian mesh (Section 4): a cell
// whose markers belong to more than one body is a collision cell, and every
// marker in it is flagged.  The markers are already grouped by spreading tile,
// so each tile's cell states live in shared memory for the duration of one
// block iteration instead of in a zeroed global array.
#include "transfer_common.cuh"

namespace mls {

// Persistent blocks walk the non-empty tiles.  For a tile: zero the state of
// its 2^(lx+ly+lz) home cells; every marker with a body index b > 0 claims
// its cell with compare-and-swap (0 -> b) and, finding another index there,
// sets the cell to -1; then every marker reads its cell: -1 flags it.  The
// occupied cells are written to `coll` when requested.  The final state of a
// cell does not depend on the order of the updates (an empty cell takes the
// first index, any second index makes it -1, and -1 is never overwritten).
__global__ void __launch_bounds__(kSpreadThreads) k_collisions(Dims D, Tiles tl, const int32_t* __restrict__ home,
                                                               const int32_t* __restrict__ perm,
                                                               const int32_t* __restrict__ items,
                                                               const int32_t* __restrict__ n_items_p,
                                                               const int32_t* __restrict__ offsets,
                                                               const int32_t* __restrict__ counts, int64_t M,
                                                               const int32_t* __restrict__ body,
                                                               int32_t* __restrict__ flag, int32_t* __restrict__ coll,
                                                               unsigned long long* __restrict__ n_colliding) {
  extern __shared__ int state[];
  const int lx = tl.l[0], ly = tl.l[1], lz = tl.l[2];
  const int TC = 1 << (lx + ly + lz);
  const int tid = threadIdx.x, lane = tid & 31;
  const int n_items = *n_items_p;
  unsigned long long found = 0;
  for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
    const int b = items[it];
    const int start = offsets[b], end = start + counts[b];
    const int bx = b % tl.nb[0], by = (b / tl.nb[0]) % tl.nb[1], bz = b / (tl.nb[0] * tl.nb[1]);
    const int ox = bx << lx, oy = by << ly, oz = bz << lz;
    for (int c = tid; c < TC; c += kSpreadThreads) state[c] = 0;
    __syncthreads();
    for (int j = start + tid; j < end; j += kSpreadThreads) {
      const int bid = body[perm[j]];
      if (bid <= 0) continue;
      int i[3];
      decode_home(home[j], D, i);
      const int c = (((i[2] - oz) << ly) + (i[1] - oy)) << lx | (i[0] - ox);
      const int old = atomicCAS(&state[c], 0, bid);
      if (old != 0 && old != bid) state[c] = -1;
    }
    __syncthreads();
    for (int j = start + tid; j < end; j += kSpreadThreads) {
      const int64_t m = perm[j];
      const int bid = body[m];
      int hit = 0;
      if (bid > 0) {
        int i[3];
        decode_home(home[j], D, i);
        hit = state[(((i[2] - oz) << ly) + (i[1] - oy)) << lx | (i[0] - ox)] == -1;
      }
      flag[m] = hit;
      found += hit;
    }
    if (coll) {
      for (int c = tid; c < TC; c += kSpreadThreads) {
        const int s = state[c];
        if (s == 0) continue;
        const int gx = ox + (c & ((1 << lx) - 1)), gy = oy + ((c >> lx) & ((1 << ly) - 1)), gz = oz + (c >> (lx + ly));
        coll[((int64_t)gz * D.n[1] + gy) * D.n[0] + gx] = s;
      }
    }
    __syncthreads();
  }
  // Markers without support: never flagged.
  const int64_t d0 = offsets[tl.nbins - 1];
  for (int64_t j = d0 + (int64_t)blockIdx.x * kSpreadThreads + tid; j < M; j += (int64_t)gridDim.x * kSpreadThreads)
    flag[perm[j]] = 0;
  if (n_colliding) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) found += __shfl_xor_sync(0xffffffffu, found, o);
    if (lane == 0 && found) atomicAdd(n_colliding, found);
  }
}

cudaError_t launch_collisions(const mls_ctx* ctx, const mls_transfer* T, const int32_t* body, int32_t* flag,
                              int32_t* coll, unsigned long long* n_colliding, cudaStream_t s) {
  if (T->M == 0) return cudaSuccess;
  const int* l = ctx->tiles.l;
  const size_t smem = (size_t)4 << (l[0] + l[1] + l[2]);
  k_collisions<<<ctx->collision_grid, kSpreadThreads, smem, s>>>(dims_of(ctx), ctx->tiles, T->home, T->perm,
                                                                 T->items, T->n_items, T->offsets, T->counts, T->M,
                                                                 body, flag, coll, n_colliding);
  return cudaGetLastError();
}

cudaError_t collision_configure(mls_ctx* ctx) {
  const int* l = ctx->tiles.l;
  const int smem = 4 << (l[0] + l[1] + l[2]);
  cudaError_t e;
  if ((e = raise_smem_limit((const void*)k_collisions, smem)) != cudaSuccess) return e;
  int per_sm = 0, sms = 0;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_collisions, kSpreadThreads, smem)) != cudaSuccess)
    return e;
  ctx->collision_grid = (per_sm > 0 ? per_sm : 1) * sms;
  return cudaSuccess;
}

}  // namespace mls
