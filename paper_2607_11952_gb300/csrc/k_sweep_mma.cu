// Phase 3 of Algorithm 1 (Eq. 3), BF16 storage of K: the fused Sinkhorn
// sweep with its row contraction on the tensor cores.
//
// One full iteration reads K once.  For a step of R <= 8 rows:
//
//   row pass     r_i  = sum_j K_ij v_j          (b update: u_i = mu_i / r_i)
//   column pass  c_j += sum_i K_ij u_i          (for the next a update)
//
// The row pass is a matrix product with one tiny dimension and runs as
// warp-level bf16 MMAs (m16n8k16) with fp32 accumulation:
//
//     D[part][row] += V[part][col] K^T[col][row]
//
// The fp32 column scaling v enters as three bfloat16 parts
// (v = hi + mid + lo: 24 significant bits, the fp32 precision) in the three
// non-zero rows of the A operand, held in shared memory for the whole
// sweep; the K tile (8 rows x 16 columns, rows past R read as zeros) is the
// B operand, read by ldmatrix straight from the ring.  K's bf16 values are
// exact, so each product is exact and only the fp32 accumulation rounds --
// the arithmetic of the CUDA-core row pass, one MMA doing the work of 128
// fused multiply-adds, and no bf16 to fp32 widening.
//
// The column pass needs one fp32 accumulator per column for the whole
// sweep; held in registers as packed fp32 pairs it stays on the CUDA cores
// (paired FMAs, each K element widened once).  Tensor-core fragments would
// need four times the registers per column.
//
// Layout and synchronisation follow the CUDA-core sweep (k_sinkhorn.cu): a
// cluster of Q CTAs owns a step of rows, CTA q its column slab of W
// columns; rows arrive by TMA bulk copies into a ring of NS stages of R
// rows; partial row sums are exchanged through distributed shared memory
// (st.async completing on the receiver's mbarrier).  A step's column pass
// follows its own exchange (no lag), so a stage is released once both
// passes are done; R (<= 8) is chosen per shape so that two stages and V
// fit beside a second CTA on the SM.  Every mbarrier wait is bounded.
#include <cuda_bf16.h>
#include <stdint.h>

#include "fa_internal.cuh"
#include "sweep_dev.cuh"

namespace fa {

namespace {

constexpr int kRmax = 8;         // rows per step at most (the MMA's n = 8)
constexpr int kMaxQm = 16;       // largest cluster
constexpr int kNXm = 4;          // exchange slots
constexpr int kMaxNSm = 4;       // largest ring

__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], uint32_t addr) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(addr));
}
// D = A B + C, m16n8k16, A rows 8..15 zero (a1 = a3 = 0)
__device__ __forceinline__ void mma_rows(float (&d)[4], uint32_t a0, uint32_t a2,
                                         uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
      "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(0u), "r"(a2), "r"(0u), "r"(b0), "r"(b1));
}
__device__ __forceinline__ void st_async_v4(uint32_t raddr, float x0, float x1, float x2,
                                            float x3, uint32_t rbar) {
  asm volatile(
      "st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.b32 [%0], {%1,%2,%3,%4}, [%5];" ::
          "r"(raddr),
      "r"(__float_as_uint(x0)), "r"(__float_as_uint(x1)), "r"(__float_as_uint(x2)),
      "r"(__float_as_uint(x3)), "r"(rbar)
      : "memory");
}

// the three bfloat16 parts of an fp32 value (x = hi + mid + lo), as raw
// 16-bit patterns
__device__ __forceinline__ void split3(float x, uint32_t& h, uint32_t& m, uint32_t& l) {
  const __nv_bfloat16 bh = __float2bfloat16_rn(x);
  const float r1 = x - __bfloat162float(bh);
  const __nv_bfloat16 bm = __float2bfloat16_rn(r1);
  const float r2 = r1 - __bfloat162float(bm);
  const __nv_bfloat16 bl = __float2bfloat16_rn(r2);
  h = __bfloat16_as_ushort(bh);
  m = __bfloat16_as_ushort(bm);
  l = __bfloat16_as_ushort(bl);
}

}  // namespace

// Shared memory: ring[NS][R][RS] | vp[3][RS] | zero[16 B] | full[kMaxNSm]
// | xbar[kNXm] | red[NW][8] | xch[kNXm][kMaxQm][8]; RS = 2 Wp + 16 bytes
// with Wp = W rounded up to 32 columns (an odd number of 16-byte units per
// row: the 8 row addresses of an ldmatrix fall in distinct banks).  vp
// holds the three bfloat16 parts of v for the slab's columns (zero past
// W); ldmatrix rows past R (K) or past the third part (V) read the zero
// chunk.  Columns W..Wp-1 of every ring row are zero-filled once and never
// written by the copies.
__host__ __device__ constexpr uint32_t mma_row_stride(int W) {
  return (uint32_t)(((W + 31) & ~31) * 2 + 16);
}
size_t sweep_mma_smem(int NS, int R, int W, int NW) {
  return (size_t)(NS * R + 3) * mma_row_stride(W) + 16 + (size_t)(kMaxNSm + kNXm) * 8 +
         (size_t)(NW * kRmax + kNXm * kMaxQm * kRmax) * sizeof(float);
}

// S: 16-byte vectors (8 columns) per thread in the column pass; NW warps;
// MINB: CTAs per SM the register budget is sized for.
template <int S, int NW, int MINB>
__global__ void __launch_bounds__(NW * 32, MINB) k_sweep_mma(
    const __nv_bfloat16* __restrict__ K, int64_t ld, int n1, int n2, int W, int NS, int R,
    const float* __restrict__ log_v, float* __restrict__ log_u, float mu,
    float log_mu, float* __restrict__ colpart, int* __restrict__ status) {
  constexpr int R8 = kRmax;
  constexpr int NT = NW * 32;
  extern __shared__ __align__(128) unsigned char smem[];
  const uint32_t RS = mma_row_stride(W);
  const uint32_t stage_bytes = (uint32_t)R * RS;
  unsigned char* vp = smem + (size_t)NS * stage_bytes;
  unsigned char* zero16 = vp + 3 * (size_t)RS;
  uint64_t* full = reinterpret_cast<uint64_t*>(zero16 + 16);
  uint64_t* xbar = full + kMaxNSm;
  float* red = reinterpret_cast<float*>(xbar + kNXm);
  float* xch = red + NW * R8;
  __shared__ int s_timeout;

  const int Q = (int)cluster_size();
  const int q = (int)cluster_rank();
  const int cg_ = blockIdx.x / Q;          // cluster = row-step group
  const int G = gridDim.x / Q;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nsteps = (n1 + R - 1) / R;
  const int T = cg_ < nsteps ? (nsteps - 1 - cg_) / G + 1 : 0;   // cluster-uniform
  const int Wp = (W + 31) & ~31;
  const int npairs = Wp / 32;              // 32-column pairs of 16-column MMA tiles
  const __nv_bfloat16* Kslab = K + (int64_t)q * W;
  const uint32_t row_bytes = (uint32_t)W * 2;
  const uint32_t xch_bytes = (uint32_t)(Q * R8 * 4);   // 8 floats from each CTA

  // zero the ring, V and the zero chunk once: the row padding (columns
  // W..Wp-1) is never written by the bulk copies, and rows past n1 in a last
  // partial step must hold finite values (they meet u = 0 in the column
  // pass).  The copies are issued by the async proxy after these
  // generic-proxy stores.
  for (uint32_t k = (uint32_t)tid; k < ((uint32_t)NS * stage_bytes + 3u * RS + 16u) / 16u;
       k += NT)
    *reinterpret_cast<uint4*>(smem + 16u * k) = make_uint4(0, 0, 0, 0);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncthreads();
  // the three bfloat16 parts of v on this slab (the row pass's A operand)
  for (int e = tid; e < W; e += NT) {
    const int64_t c = (int64_t)q * W + e;
    const float v = c < n2 ? expf(log_v[c]) : 0.f;
    uint32_t h, m, l;
    split3(v, h, m, l);
    reinterpret_cast<uint16_t*>(vp)[e] = (uint16_t)h;
    reinterpret_cast<uint16_t*>(vp + RS)[e] = (uint16_t)m;
    reinterpret_cast<uint16_t*>(vp + 2 * RS)[e] = (uint16_t)l;
  }
  if (tid == 0) {
    for (int s = 0; s < NS; ++s) mbar_init(smem_u32(&full[s]), 1);
    for (int s = 0; s < kNXm; ++s) mbar_init(smem_u32(&xbar[s]), 1);
    fence_mbar_init();
    s_timeout = 0;
    if (Q > 1)
      for (int t = 0; t < min(kNXm, T); ++t) mbar_expect_tx(smem_u32(&xbar[t]), xch_bytes);
  }
  __syncthreads();
  if (Q > 1) {   // every CTA's barriers exist before any remote store
    cluster_arrive();
    cluster_wait();
  }

  // column pass: this thread owns the 16-byte vectors tid + NT s of each
  // ring row (columns 2k, 2k + 1 of a vector as one packed fp32 pair)
  f2_t acc[S][4];
  uint32_t voff[S];
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const int e0 = (s * NT + tid) * 8;
    // a vector past the slab edge reads the slab's last vector; its
    // accumulators are never stored
    voff[s] = (uint32_t)((e0 < W ? e0 : W - 8) * 2);
#pragma unroll
    for (int k = 0; k < 4; ++k) acc[s][k] = pk2(0.f, 0.f);
  }
  // vectors s < S-1 are inside the slab for every thread; the last one only
  // for the first warps: skip it warp-uniformly where no lane has one
  const bool last_ok = ((S - 1) * NT + warp * 32) * 8 < W;

  // ldmatrix row addresses: row lane & 7, the 8-column group lane >> 3 of a
  // 32-column pair; K rows past R and V rows past the third part read zeros
  const uint32_t ring_s = smem_u32(smem);
  const uint32_t zero_s = smem_u32(zero16);
  const int lrow = lane & 7;
  const uint32_t col_off = 16u * (uint32_t)(lane >> 3);
  const bool krow_ok = lrow < R;
  const uint32_t v_addr = lrow < 3 ? smem_u32(vp) + (uint32_t)lrow * RS + col_off : zero_s;
  const uint32_t v_step = lrow < 3 ? 64u : 0u;
  const uint32_t kstep = krow_ok ? 64u : 0u;

  int issued = 0;   // meaningful in thread 0 only
  auto issue = [&](int t, int stage) {
    const int row0 = (cg_ + t * G) * R;
    const int nrows = min(R, n1 - row0);
    const uint32_t mb = smem_u32(&full[stage]);
    mbar_expect_tx(mb, (uint32_t)nrows * row_bytes);
    for (int r = 0; r < nrows; ++r)
      bulk_g2s(ring_s + (uint32_t)stage * stage_bytes + (uint32_t)r * RS,
               Kslab + (int64_t)(row0 + r) * ld, row_bytes, mb);
  };
  if (tid == 0) {
    for (int t = 0; t < min(NS, T); ++t) issue(t, t);
    issued = min(NS, T);
  }

  bool dead = false;
  int stage = 0;
  uint32_t ph = 0;
  for (int t = 0; t < T; ++t) {
    if (!dead && !mbar_wait_bounded(smem_u32(&full[stage]), ph)) {
      atomicOr(status, ST_TIMEOUT);
      s_timeout = 1;
    }
    const int row0 = (cg_ + t * G) * R;
    const uint32_t sring = ring_s + (uint32_t)stage * stage_bytes;
    const uint32_t kaddr = krow_ok ? sring + (uint32_t)lrow * RS + col_off : zero_s;

    // -------- row pass (tensor cores): partial row sums of this warp's
    // 32-column pairs; lane (g, tq), g < 3, accumulates part g of rows
    // 2 tq and 2 tq + 1
    float dr[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
#pragma unroll 2
    for (int p = warp; p < npairs; p += NW) {
      uint32_t a[4], b[4];
      ldsm_x4(a, v_addr + v_step * (uint32_t)p);
      ldsm_x4(b, kaddr + kstep * (uint32_t)p);
      mma_rows(dr[0], a[0], a[1], b[0], b[1]);
      mma_rows(dr[1], a[2], a[3], b[2], b[3]);
    }
    float x0 = dr[0][0] + dr[1][0];
    float x1 = dr[0][1] + dr[1][1];
    {   // add the three parts (lanes +4 and +8 hold parts 1 and 2)
      const float y0 = __shfl_down_sync(0xffffffffu, x0, 4);
      const float y1 = __shfl_down_sync(0xffffffffu, x1, 4);
      const float z0 = __shfl_down_sync(0xffffffffu, x0, 8);
      const float z1 = __shfl_down_sync(0xffffffffu, x1, 8);
      x0 = (x0 + y0) + z0;
      x1 = (x1 + y1) + z1;
    }
    if (lane < 4) {
      red[warp * R8 + 2 * lane] = x0;
      red[warp * R8 + 2 * lane + 1] = x1;
    }
    __syncthreads();
    // -------- exchange the CTA's partial row sums within the cluster
    if (Q > 1 && warp == 0) {
      float rs = 0.f;
#pragma unroll
      for (int w = 0; w < NW; ++w) rs += red[w * R8 + (lane & 7)];
      const int half = lane / Q, dst = lane - half * Q;    // lane < 2 Q sends
      const float p0 = __shfl_sync(0xffffffffu, rs, (4 * half + 0) & 7);
      const float p1 = __shfl_sync(0xffffffffu, rs, (4 * half + 1) & 7);
      const float p2 = __shfl_sync(0xffffffffu, rs, (4 * half + 2) & 7);
      const float p3 = __shfl_sync(0xffffffffu, rs, (4 * half + 3) & 7);
      if (lane < 2 * Q) {
        const uint32_t slot = smem_u32(xch + ((t % kNXm) * kMaxQm + q) * R8 + 4 * half);
        const uint32_t bar = smem_u32(&xbar[t % kNXm]);
        st_async_v4(map_cluster(slot, (uint32_t)dst), p0, p1, p2, p3,
                    map_cluster(bar, (uint32_t)dst));
      }
    }
    if (Q > 1 && !dead &&
        !mbar_wait_bounded(smem_u32(&xbar[t % kNXm]), (uint32_t)((t / kNXm) & 1))) {
      atomicOr(status, ST_TIMEOUT);
      s_timeout = 1;
    }
    // -------- full row sums (CTA order, identical in every CTA) and u;
    // lane r (mod 8) holds row r of the step
    float rsum = 0.f;
    if (Q > 1) {
      const float* xs = xch + (t % kNXm) * kMaxQm * R8 + (lane & 7);
      for (int c = 0; c < Q; ++c) rsum += xs[c * R8];
    } else {
#pragma unroll
      for (int w = 0; w < NW; ++w) rsum += red[w * R8 + (lane & 7)];
    }
    const int row = row0 + (lane & 7);
    float u = 0.f;
    if ((lane & 7) < R && row < n1) {
      if (rsum > 0.f && isfinite(rsum)) {
        u = mu / rsum;
        if (!isfinite(u)) {
          u = 0.f;
          if (warp == 0 && lane < 8) atomicOr(status, ST_NUMERIC);
        }
      } else if (warp == 0 && lane < 8) {
        atomicOr(status, ST_NUMERIC);
      }
      if (q == 0 && warp == 0 && lane < 8) log_u[row] = log_mu - logf(rsum);
    }
    // -------- column pass (CUDA cores): acc_j += K_rj u_r
    for (int r = 0; r < R; ++r) {
      const float ur = __shfl_sync(0xffffffffu, u, r);
      const f2_t u2 = pk2(ur, ur);
      const uint32_t rbase = sring + (uint32_t)r * RS;
#pragma unroll
      for (int s = 0; s < S; ++s) {
        if (s + 1 < S || last_ok) {
          f2_t f[4];
          pairs(lds128a(rbase + voff[s]), f, __nv_bfloat16());
#pragma unroll
          for (int k = 0; k < 4; ++k) acc[s][k] = ffma2(u2, f[k], acc[s][k]);
        }
      }
    }
    __syncthreads();   // stage, red and exchange slot consumed
    dead = s_timeout != 0;
    if (tid == 0) {
      if (Q > 1 && t + kNXm < T) mbar_expect_tx(smem_u32(&xbar[t % kNXm]), xch_bytes);
      if (!dead && t + NS < T) {
        issue(t + NS, stage);
        issued = t + NS + 1;
      }
    }
    if (++stage == NS) {
      stage = 0;
      ph ^= 1u;
    }
  }
  // after a timeout, wait (bounded) for copies still in flight into the ring
  if (tid == 0 && dead) {
    for (int t = max(0, issued - NS); t < issued; ++t)
      mbar_wait_bounded(smem_u32(&full[t % NS]), (uint32_t)((t / NS) & 1));
  }
  if (Q > 1) {   // no CTA leaves while a peer may still address its memory
    cluster_arrive();
    cluster_wait();
  }
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const int e0 = (s * NT + tid) * 8;
    if (e0 < W) {
      float* dst = colpart + (int64_t)cg_ * ld + (int64_t)q * W + e0;
      const float2 a = upk2(acc[s][0]), b = upk2(acc[s][1]);
      const float2 c = upk2(acc[s][2]), d = upk2(acc[s][3]);
      *reinterpret_cast<float4*>(dst) = make_float4(a.x, a.y, b.x, b.y);
      *reinterpret_cast<float4*>(dst + 4) = make_float4(c.x, c.y, d.x, d.y);
    }
  }
}

// Shapes instantiated: (S, NW, MINB).
void* sweep_mma_kernel(int S, int NW, int MINB) {
#define FA_M(SS, N, B) \
  if (S == SS && NW == N && MINB == B) return reinterpret_cast<void*>(&k_sweep_mma<SS, N, B>);
  FA_M(1, 4, 2) FA_M(2, 4, 2) FA_M(3, 4, 2) FA_M(4, 4, 2) FA_M(5, 4, 2) FA_M(6, 4, 2)
  FA_M(1, 8, 1) FA_M(2, 8, 1) FA_M(3, 8, 1) FA_M(4, 8, 1) FA_M(5, 8, 1) FA_M(6, 8, 1)
  FA_M(7, 8, 1) FA_M(8, 8, 1)
#undef FA_M
  return nullptr;
}

}  // namespace fa
