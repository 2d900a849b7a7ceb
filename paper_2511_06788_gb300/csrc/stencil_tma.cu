// Step 1 of §4.1 on 3-D grids, FP32 blocks: the direction kernel of a
// conjugate-gradient iteration with its 7-point stencil operand staged in shared
// memory by TMA bulk-tensor loads.
//
// A block (n x ld floats, row-major, point index ix + nx (iy + ny iz)) is the
// 4-D tensor [nz][ny][nx][ld], cut into columns of 8 x 8 points by 32 matrix
// columns through all z.  A persistent CTA marches one column (or a z-slab of
// one) in +z at a time, in lockstep with the CTAs on the neighbouring columns.
// Per plane the CTA loads the 10 x 10 x 32 box around
// its tile (a one-point halo; TMA fills coordinates outside the grid with zeros,
// which is the Dirichlet boundary) into a ring of shared-memory slots.  A thread
// owns one float4 of two y-adjacent points: it keeps the centre values of planes
// z-1, z, z+1 in registers and reads its x and y neighbours from the box of
// plane z, so every element is fetched from L2 about 1.6 times (halo) instead of
// seven.
//
//   k_cg_tma<M_P_FIRST / M_P>:  Pn = R (+ beta Po), the R box converted in place;
//                     part = Pn . (H + sigma) Pn per column.
//   k_cg_tma<M_QUAD>: the energy sums part = (X . (H + sigma) X, X . X).
// V of the next plane to compute is loaded into registers one plane ahead, so
// its latency overlaps the wait for the next box.
//
// Partial sums: per thread in FP32, then over threads and warps in FP64 in a
// fixed order; one row of `part` per CTA (zero for the chunks it does not touch).
// Every mbarrier wait gives up after two seconds: the CTA then sets the error
// flag, waits (bounded) for the copies it has in flight and returns.
#include <mutex>

#include "common.cuh"
#include "kernels.cuh"
#include "tma.cuh"

namespace opevo {

namespace {

constexpr int kTX = 8, kTY = 8, kPC = 32;  // tile: 8 x 8 points x 32 columns
constexpr int kBX = kTX + 2, kBY = kTY + 2;
constexpr int kV = kPC / 4;                 // float4 per point and chunk
constexpr int kHaloV = kBX * kBY * kV;      // float4 of a halo box (800)
constexpr int kHaloBytes = kHaloV * 16;     // 12800
constexpr int kThreads = 256;
constexpr uint64_t kWaitNs = 2000000000ull;

// Modes of the plane-marching kernel (the box loaded per plane, what is computed):
//   M_P_FIRST  R box:         Pn = R;            part = Pn . A Pn
//   M_P        R and Po box:  Pn = R + beta Po;  part = Pn . A Pn
//   M_QUAD     X box:         part = (X . A X, X . X)
// with A = H + sigma (the shift of the geometry passed in).
enum { M_P_FIRST = 0, M_P = 1, M_QUAD = 2 };

template <int MODE> struct Slot {
  static constexpr int bytes = MODE == M_P ? 2 * kHaloBytes : kHaloBytes;
  static constexpr int ncomp = MODE >= M_QUAD ? 2 : 1;  // partial sums per column
  // ring depth (up to ns - 1 planes in flight): 4 slots of two boxes or 8 of one box,
  // about 100 KB either way, two CTAs per SM
  static constexpr int ns = MODE == M_P ? 4 : 8;
};

template <int MODE, int NS> constexpr int smem_bytes() {
  return 128 + NS * Slot<MODE>::bytes + 2 * NS * 8;
}

// Work items: (slab, column), column = chunk * ntiles + tile; slab s of S covers
// planes [nz s / S, nz (s + 1) / S).  Item it = s * ncols + column; CTA b takes
// items b, b + G, b + 2G, ... so that at any time the CTAs march neighbouring
// columns through the same planes and the halo rows one CTA loads are still in
// L2 when its neighbour loads them as its own.  Load j of an item brings plane
// za - 1 + j, j = 0 .. m + 1 (m planes computed).
struct Cursor {
  long long it;
  int za, m, j, chunk, x0, y0;
  __device__ __forceinline__ void set_item(const CgTmaGeom &tg) {
    const int ncols = tg.nch * tg.ntx * tg.nty, ntiles = tg.ntx * tg.nty;
    const int sl = (int)(it / ncols), col = (int)(it % ncols);
    chunk = col / ntiles;
    const int t = col % ntiles;
    x0 = (t % tg.ntx) * kTX;
    y0 = (t / tg.ntx) * kTY;
    za = (int)((long long)tg.nz * sl / tg.slabs);
    m = (int)((long long)tg.nz * (sl + 1) / tg.slabs) - za;
  }
  __device__ __forceinline__ void start(const CgTmaGeom &tg) {
    it = blockIdx.x;
    j = 0;
    if (valid(tg)) set_item(tg);
  }
  __device__ __forceinline__ bool valid(const CgTmaGeom &tg) const { return it < tg.items; }
  __device__ __forceinline__ void next(const CgTmaGeom &tg) {
    if (++j == m + 2) {
      it += gridDim.x;
      j = 0;
      if (valid(tg)) set_item(tg);
    }
  }
};

// Thread 0: start load number L (slot L % NS) for the cursor's next plane.
template <int MODE, int NS>
__device__ __forceinline__ void issue(const CgTmaGeom &tg, const Cursor &cur, long long L,
                                      unsigned char *slots, uint64_t *bars, const CUtensorMap *mA,
                                      const CUtensorMap *mB) {
  const int plane = cur.za - 1 + cur.j;
  const int slot = (int)(L % NS);
  unsigned char *s = slots + slot * Slot<MODE>::bytes;
  uint64_t *bar = bars + slot;
  if (plane < 0 || plane >= tg.nz) {  // outside the grid: zero plane, no copy
    tma::bar_arrive(bar);
    return;
  }
  tma::bar_expect(bar, Slot<MODE>::bytes);
  const int c0 = cur.chunk * kPC;
  tma::load_4d(s, mA, c0, cur.x0 - 1, cur.y0 - 1, plane, bar);
  if (MODE == M_P) tma::load_4d(s + kHaloBytes, mB, c0, cur.x0 - 1, cur.y0 - 1, plane, bar);
}

__device__ __forceinline__ float4 f4_zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }

// Barrier among the compute warps only (the producer warp does not take part).
__device__ __forceinline__ void compute_sync() {
  asm volatile("bar.sync 1, %0;" ::"n"(kThreads) : "memory");
}

// Add acc, summed over the 32 threads sharing its columns (FP64, fixed order), to
// prow[chunk * 32 + c]; resets acc.  Compute warps only.
__device__ __forceinline__ void flush(float *acc, int chunk, int ld, double *prow,
                                      double (*red)[kPC]) {
  const int tid = threadIdx.x, lane = tid & 31, wp = tid >> 5;
  double d[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    d[k] = (double)acc[k];
    d[k] += __shfl_xor_sync(0xffffffffu, d[k], 8);
    d[k] += __shfl_xor_sync(0xffffffffu, d[k], 16);
    acc[k] = 0.f;
  }
  if (lane < kV) {
#pragma unroll
    for (int k = 0; k < 4; ++k) red[wp][lane * 4 + k] = d[k];
  }
  compute_sync();
  if (tid < kPC) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < kThreads / 32; ++w) s += red[w][tid];
    const int col = chunk * kPC + tid;
    if (col < ld) prow[col] += s;
  }
  compute_sync();
}

// Warps 0-7 compute; warp 8 (one lane) produces: it refills a slot with the next
// plane as soon as every compute warp has released it ("empty" barrier, 8
// arrivals), and the compute warps wait for the data on the slot's "full"
// barrier (1 arrival + the copy's bytes).
template <int MODE, int NS>
__global__ void __launch_bounds__(kThreads + 32, 2)
    k_cg_tma(CgTmaGeom tg, const float *__restrict__ Vt, const __grid_constant__ CUtensorMap mA,
             const __grid_constant__ CUtensorMap mB, float *__restrict__ out,
             const double *__restrict__ beta, const int *nact_prev, double *__restrict__ part,
             int *err) {
  if (nact_prev && *nact_prev == 0) return;
  constexpr int SB = Slot<MODE>::bytes;
  constexpr int NC = Slot<MODE>::ncomp;
  constexpr bool FIRST = MODE != M_P;  // no P_old box to fold in
  extern __shared__ unsigned char dsm[];
  unsigned char *slots =
      (unsigned char *)(((uintptr_t)dsm + 127) & ~(uintptr_t)127);
  uint64_t *full = (uint64_t *)(slots + NS * SB);
  uint64_t *empty = full + NS;
  __shared__ double red[kThreads / 32][kPC];
  __shared__ volatile int s_abort;

  const int tid = threadIdx.x;
  const int ld = tg.ld;
  double *prow = part + (long long)blockIdx.x * NC * ld;  // this CTA's partials (flush adds)
  for (int col = tid; col < NC * ld; col += kThreads + 32) prow[col] = 0.0;
  if (tid == 0) {
    for (int s = 0; s < NS; ++s) {
      tma::bar_init(full + s, 1);
      tma::bar_init(empty + s, kThreads / 32);
    }
    s_abort = 0;
    tma::fence_bar_init();
  }
  __syncthreads();

  if (tid >= kThreads) {  // producer warp
    if (tid != kThreads) return;
    Cursor prod;
    prod.start(tg);
    long long l = 0;
    for (; prod.valid(tg); ++l, prod.next(tg)) {
      const int slot = (int)(l % NS);
      if (l >= NS && !tma::bar_wait(empty + slot, (uint32_t)((l / NS - 1) & 1), kWaitNs)) {
        s_abort = 1;
        atomicExch(err, 1);
      }
      if (s_abort) break;
      issue<MODE, NS>(tg, prod, l, slots, full, &mA, &mB);
    }
    // copies still in flight land before the CTA may exit (only the last NS can be)
    if (s_abort)
      for (long long k = (l > NS ? l - NS : 0); k < l; ++k)
        tma::bar_wait(full + (int)(k % NS), (uint32_t)((k / NS) & 1), kWaitNs);
    return;
  }

  const int c4 = tid & 7, xl = (tid >> 3) & 7, ya = (tid >> 6) * 2;
  Cursor cons;
  cons.start(tg);
  long long L = 0;
  float4 cp[2] = {f4_zero(), f4_zero()}, cc[2] = {f4_zero(), f4_zero()};
  float vc[2] = {0.f, 0.f};  // V of the next plane to compute
  float acc[NC][4] = {};
  float cf[4] = {0.f, 0.f, 0.f, 0.f};
  int chunk = -1;
  const float cx = tg.cx, cy = tg.cy, cz = tg.cz;

  while (cons.valid(tg)) {
    const Cursor w = cons;
    const int plane = w.za - 1 + w.j;
    const int m = w.m;
    if (w.chunk != chunk) {
      chunk = w.chunk;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int col = chunk * kPC + c4 * 4 + k;
        cf[k] = (!FIRST && col < ld) ? (float)beta[col] : 0.f;
      }
    }
    const int slot = (int)(L % NS);
    unsigned char *s = slots + slot * SB;
    const bool in_range = plane >= 0 && plane < tg.nz;
    if (!tma::bar_wait(full + slot, (uint32_t)((L / NS) & 1), kWaitNs)) {
      s_abort = 1;
      atomicExch(err, 1);
    }
    if (MODE == M_P && in_range) {  // Pn = R + beta Po over the whole box
      float4 *r = (float4 *)s;
      const float4 *po = (const float4 *)(s + kHaloBytes);
      for (int e = tid; e < kHaloV; e += kThreads) {  // e % 8 == c4
        float4 a = r[e];
        const float4 b = po[e];
        a.x += cf[0] * b.x;
        a.y += cf[1] * b.y;
        a.z += cf[2] * b.z;
        a.w += cf[3] * b.w;
        r[e] = a;
      }
    }
    compute_sync();
    if (s_abort) break;
    float4 cn[2];
    {
      const float4 *box = (const float4 *)s;
#pragma unroll
      for (int i = 0; i < 2; ++i)
        cn[i] = in_range ? box[((ya + i + 1) * kBX + xl + 1) * kV + c4] : f4_zero();
    }
    const int x = w.x0 + xl;
    const int col = chunk * kPC + c4 * 4;
    if (w.j >= 2) {  // plane zc = plane - 1 is complete: compute it
      const int zc = plane - 1;
      const float4 *hb = (const float4 *)(slots + (int)((L - 1) % NS) * SB);
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const int yl = ya + i, y = w.y0 + yl;
        const int bi = ((yl + 1) * kBX + xl + 1) * kV + c4;
        const float4 l = hb[bi - kV], r = hb[bi + kV];
        const float4 dn = (i == 0) ? hb[bi - kBX * kV] : cc[0];
        const float4 up = (i == 1) ? hb[bi + kBX * kV] : cc[1];
        if (!(x < tg.nx && y < tg.ny && col < ld)) continue;
        const long long pt = ((long long)zc * tg.ny + y) * tg.nx + x;
        const float d = vc[i] + tg.shift;
        const float4 c = cc[i];
        float4 q;
        q.x = d * c.x - cx * (l.x + r.x) - cy * (dn.x + up.x) - cz * (cp[i].x + cn[i].x);
        q.y = d * c.y - cx * (l.y + r.y) - cy * (dn.y + up.y) - cz * (cp[i].y + cn[i].y);
        q.z = d * c.z - cx * (l.z + r.z) - cy * (dn.z + up.z) - cz * (cp[i].z + cn[i].z);
        q.w = d * c.w - cx * (l.w + r.w) - cy * (dn.w + up.w) - cz * (cp[i].w + cn[i].w);
        if (MODE != M_QUAD) *reinterpret_cast<float4 *>(out + pt * ld + col) = c;
        acc[0][0] += c.x * q.x;
        acc[0][1] += c.y * q.y;
        acc[0][2] += c.z * q.z;
        acc[0][3] += c.w * q.w;
        if (MODE == M_QUAD) {
          acc[NC - 1][0] += c.x * c.x;
          acc[NC - 1][1] += c.y * c.y;
          acc[NC - 1][2] += c.z * c.z;
          acc[NC - 1][3] += c.w * c.w;
        }
      }
    }
    // slot L - 1 is no longer read by this warp: release it to the producer
    if (L >= 1) {
      tma::fence_proxy_async();
      __syncwarp();
      if ((tid & 31) == 0) tma::bar_arrive(empty + (int)((L - 1) % NS));
    }
    // V of the plane computed next iteration (this load's plane), fetched one
    // iteration ahead so that its latency overlaps the pipeline wait
    if (w.j >= 1 && w.j <= m) {
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const int y = w.y0 + ya + i;
        const long long pt = ((long long)plane * tg.ny + y) * tg.nx + x;
        vc[i] = (x < tg.nx && y < tg.ny) ? __ldg(Vt + pt) : 0.f;
      }
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      cp[i] = cc[i];
      cc[i] = cn[i];
    }
    const bool last = w.j == m + 1;
    cons.next(tg);
    ++L;
    if (last) {
      const int nc = cons.valid(tg) ? cons.chunk : -1;
      if (nc != chunk)
        for (int q = 0; q < NC; ++q) flush(acc[q], chunk, ld, prow + q * ld, red);
    }
  }
}


// Resident CTAs per SM of the kernel for MODE on the current device; the first call on a
// device also sets the kernel's shared-memory attribute there (attributes are per device).
template <int MODE>
int resident_ctas() {
  constexpr int kMaxDev = 64;
  static int cached[kMaxDev] = {};
  static std::mutex mu;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) {
    cudaGetLastError();
    dev = 0;
  }
  std::lock_guard<std::mutex> lk(mu);
  if (cached[dev] < 1) {
    constexpr int NS = Slot<MODE>::ns;
    const int bytes = smem_bytes<MODE, NS>();
    cudaFuncSetAttribute(k_cg_tma<MODE, NS>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cg_tma<MODE, NS>, kThreads + 32,
                                                      bytes) != cudaSuccess ||
        per_sm < 1)
      per_sm = 1;
    cached[dev] = per_sm;
  }
  return cached[dev];
}

// Geometry and persistent grid shared by every mode (so that all of them write the
// same number of partial rows).  One wave of resident CTAs of the largest mode:
// whole columns (S = 1) when there are at least as many columns as CTAs, else each
// column cut into S z-slabs.
void plan_geometry(const Geom &g, double sigma, int ld, CgTmaGeom *tg, int *grid) {
  tg->nx = g.nx;
  tg->ny = g.ny;
  tg->nz = g.nz;
  tg->ld = ld;
  tg->ntx = (g.nx + kTX - 1) / kTX;
  tg->nty = (g.ny + kTY - 1) / kTY;
  tg->nch = (ld + kPC - 1) / kPC;
  tg->shift = (float)(g.cdiag + sigma);
  tg->cx = (float)g.c[0];
  tg->cy = (float)g.c[1];
  tg->cz = (float)g.c[2];
  int per_sm = resident_ctas<M_P>();
  const int others[2] = {resident_ctas<M_P_FIRST>(), resident_ctas<M_QUAD>()};
  for (int o : others) per_sm = o < per_sm ? o : per_sm;
  const long long cap = (long long)num_sms() * per_sm;
  const long long ncols = (long long)tg->nch * tg->ntx * tg->nty;
  long long S = ncols < cap ? cap / ncols : 1;
  if (S > g.nz) S = g.nz;
  tg->slabs = (int)S;
  tg->items = ncols * S;
  *grid = (int)(tg->items < cap ? tg->items : cap);
}

op_status halo_map(const Geom &g, int ld, const float *X, CUtensorMap *map) {
  const uint64_t dims[4] = {(uint64_t)ld, (uint64_t)g.nx, (uint64_t)g.ny, (uint64_t)g.nz};
  const uint32_t halo[4] = {kPC, kBX, kBY, 1};
  return tma_map_4d_f32(map, X, dims, halo);
}

}  // namespace

bool cg_tma_eligible(const Geom &g, int ld, const void *R, const void *P, const void *Q) {
  const uintptr_t a = (uintptr_t)R | (uintptr_t)P | (uintptr_t)Q;
  return g.dim == 3 && ld >= kPC && ld % 4 == 0 && g.nz >= 3 && (a & 15) == 0;
}

op_status cg_tma_prepare(const Geom &g, double sigma, int ld, const float *R, const float *P,
                         const float *Q, CgTmaPlan *plan) {
  plan_geometry(g, sigma, ld, &plan->tg, &plan->grid);
  OP_TRY(halo_map(g, ld, R, &plan->halo[0]));
  OP_TRY(halo_map(g, ld, P, &plan->halo[1]));
  OP_TRY(halo_map(g, ld, Q, &plan->halo[2]));
  return OP_OK;
}

op_status cg_tma_p(const CgTmaPlan &plan, bool first, int po, float *Pn, const float *Vt,
                   const double *beta, const int *nact_prev, double *part, int *err,
                   cudaStream_t st) {
  const CUtensorMap &mR = plan.halo[0];
  const CUtensorMap &mPo = plan.halo[po == 0 ? 1 : 2];
  if (first)
    k_cg_tma<M_P_FIRST, 8><<<plan.grid, kThreads + 32, smem_bytes<M_P_FIRST, 8>(), st>>>(
        plan.tg, Vt, mR, mPo, Pn, beta, nact_prev, part, err);
  else
    k_cg_tma<M_P, 4><<<plan.grid, kThreads + 32, smem_bytes<M_P, 4>(), st>>>(
        plan.tg, Vt, mR, mPo, Pn, beta, nact_prev, part, err);
  count_launch();
  OP_LAUNCH("k_cg_tma");
  return OP_OK;
}

op_status tma_quad(const Geom &g, double sigma, int ld, const float *Vt, const float *X,
                   double *part, int *err, int *grid, cudaStream_t st) {
  CgTmaGeom tg;
  plan_geometry(g, sigma, ld, &tg, grid);
  CUtensorMap mX;
  OP_TRY(halo_map(g, ld, X, &mX));
  k_cg_tma<M_QUAD, 8><<<*grid, kThreads + 32, smem_bytes<M_QUAD, 8>(), st>>>(
      tg, Vt, mX, mX, nullptr, nullptr, nullptr, part, err);
  count_launch();
  OP_LAUNCH("k_cg_tma<quad>");
  return OP_OK;
}

// ---------------------------------------------------------------------------
// Tensor-map encoding through the driver entry point (no libcuda link needed).
// ---------------------------------------------------------------------------
namespace {
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  });
  return fn;
}
}  // namespace

op_status tma_map_4d_f32(CUtensorMap *map, const void *base, const uint64_t dims[4],
                         const uint32_t box[4]) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) {
    set_error("cuTensorMapEncodeTiled is not available from the driver");
    return OP_ERR_CUDA;
  }
  if (((uintptr_t)base & 15) != 0 || (dims[0] * 4) % 16 != 0 || (box[0] * 4) % 16 != 0) {
    set_error("tensor map: base, row pitch or box row not 16-byte aligned");
    return OP_ERR_ARG;
  }
  cuuint64_t gd[4] = {dims[0], dims[1], dims[2], dims[3]};
  cuuint64_t gs[3] = {dims[0] * 4, dims[0] * dims[1] * 4, dims[0] * dims[1] * dims[2] * 4};
  cuuint32_t bx[4] = {box[0], box[1], box[2], box[3]};
  cuuint32_t es[4] = {1, 1, 1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<void *>(base), gd, gs, bx,
                  es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed (CUresult %d)", (int)r);
    return OP_ERR_CUDA;
  }
  return OP_OK;
}

op_status tma_map_2d_f32_sw128(CUtensorMap *map, const void *base, uint64_t inner, uint64_t outer,
                               uint32_t box_outer) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) {
    set_error("cuTensorMapEncodeTiled is not available from the driver");
    return OP_ERR_CUDA;
  }
  if (((uintptr_t)base & 15) != 0 || (inner * 4) % 16 != 0) {
    set_error("tensor map: base or row pitch not 16-byte aligned");
    return OP_ERR_ARG;
  }
  cuuint64_t gd[2] = {inner, outer};
  cuuint64_t gs[1] = {inner * 4};
  cuuint32_t bx[2] = {32, box_outer};
  cuuint32_t es[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void *>(base), gd, gs, bx,
                  es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed (CUresult %d)", (int)r);
    return OP_ERR_CUDA;
  }
  return OP_OK;
}

op_status tma_map_3d_bf16_sw(CUtensorMap *map, const void *base, uint64_t inner,
                             uint64_t rows, uint64_t planes, uint32_t box_rows, uint32_t box_k) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) {
    set_error("cuTensorMapEncodeTiled is not available from the driver");
    return OP_ERR_CUDA;
  }
  if (((uintptr_t)base & 15) != 0 || (inner * 2) % 16 != 0 || box_rows < 1 || box_rows > 256 ||
      (box_k != 16 && box_k != 32)) {
    set_error("tensor map: base or row pitch not 16-byte aligned, or bad box");
    return OP_ERR_ARG;
  }
  cuuint64_t gd[3] = {inner, rows, planes};
  cuuint64_t gs[2] = {inner * 2, inner * rows * 2};
  cuuint32_t bx[3] = {box_k, box_rows, 1};
  cuuint32_t es[3] = {1, 1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void *>(base), gd, gs, bx,
                  es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  box_k == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed (CUresult %d)", (int)r);
    return OP_ERR_CUDA;
  }
  return OP_OK;
}

}  // namespace opevo
