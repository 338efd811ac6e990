// Batched gradient iterations on the packed symmetric P (Eq. 4, Eq. 6,
// Eq. 12/13) and the per-chunk cost (Eq. 5, Eq. 9) — the ptSNE hot loop.
//
// One persistent launch runs every iteration of every chunk of an epoch.  A
// chunk is owned by a cluster of K blocks (K = 1, 2 or 4); the chunk's map
// lives in every block's shared memory and each block takes a contiguous
// K-th of the chunk's stored tiles (stored row block by row block).  Within
// a block every warp evaluates whole tiles: warp w of W takes a contiguous
// W-th of the block's share (P tiles of 4 KB, stored once per unordered pair
// of 32-row blocks), the same piece in every pass, and owns one shared tile
// buffer.  For each tile it waits for its own copy (cp.async, each lane
// copying the eight 16-byte pieces of P it will read back), reads the tile
// into registers, starts the copy of its next tile into the buffer, and then
// evaluates the tile from registers: the next copy has a whole tile's
// arithmetic to land.  No producer warp, no barrier between warps and no
// spin-wait in the tile loop.
//   - an off-diagonal tile (rows a, columns b) is evaluated once per unordered
//     pair: w = 1 / (1 + |y_i - y_j|^2) and the terms p_ij w (y_i - y_j) of
//     A and w^2 (y_i - y_j) of R go to row i and, negated, to row j (column
//     sums travel around rings of lanes, see the tile evaluation below), and
//     2 w to Z; a diagonal tile holds both orders and is evaluated row-wise.
//     For 2-D maps a warp keeps the row sums of its current row block in
//     registers across its tiles and adds them to the accumulators when the
//     row block changes;
//     So P is read once per unordered pair (2 bytes per ordered pair) and w is
//     computed once per unordered pair.  Packed f32x2 arithmetic for 2-D
//     maps; the sums are merged into shared-memory accumulators with atomic
//     adds;
//   - then Z = sum_i Z_i (FP64, over the cluster through distributed shared
//     memory), dC/dy_i = 4 (A_i - R_i / Z) (Eq. 6), and the update of each
//     block's slice of rows, broadcast to every block's copy of the map.
#include <float.h>

#include "ptsne_internal.cuh"

namespace ptsne {

namespace {
// Padding rows (z <= i < 32 nb) sit at (i - z + 1) * kPad on every axis: any
// pair with a padding row is >= 1e18 apart, so w <= 1e-36 (or 0 once the
// square overflows) and p = 0, and padding rows can be processed like real
// ones without changing A, R or Z (their own updates are never written).
constexpr float kPad = 1e18f;
constexpr float kLn2f = 0.69314718055994531f;
constexpr int kStaticSmem = 2048;               // bound on the kernel's static shared memory
constexpr int kMaxWarps = 24;                   // warps per block (the builds run at most 21)
}  // namespace

struct IterArgs {
    const float* P2;            // packed tiles of all chunks
    const int64_t* ptile_off;   // n_chunks: first tile of each chunk
    Layout L;
    float* Yc;                  // n x od map, permuted order (in/out)
    float* vel;
    float* gains;
    float* gradp;               // optional: gradient at the input map (permuted order)
    double* Zc;                 // optional: Z of the last gradient pass, per chunk
    double* cost_chunk;         // cost pass: {KL, normalised cost} per chunk
    int iters;                  // gradient passes
    int cost_pass;              // 1: one cost pass after the gradient passes
    Optim opt;
    int* queue;                 // chunk work queue (zeroed before launch)
    int zcap;                   // rows of the shared map / accumulators (multiple of 32)
    int acc_rows;               // rows of one block's accumulators: zcap, or, when the deterministic
                                // build splits its sums over a cluster of K > 1 blocks, ceil(zcap / K)
                                // rounded up to 32 (each block holds the sums of the rows it updates)
};

// ---------------------------------------------------------------- PTX helpers

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// 16-byte copy global -> shared, completed by cp.async.wait_group; cached in
// L2 only (P is read once per pass).
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ uint32_t cl_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cl_size() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ void cl_barrier() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// block barrier, or cluster barrier when the chunk is shared by several blocks
__device__ __forceinline__ void sync_owner(uint32_t K) {
    if (K > 1) cl_barrier();
    else __syncthreads();
}
__device__ __forceinline__ uint32_t map_rank(uint32_t addr, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}
__device__ __forceinline__ float ld_cl_f32(uint32_t a) {
    float v;
    asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ double ld_cl_f64(uint32_t a) {
    double v;
    asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ long long ld_cl_s64(uint32_t a) {
    long long v;
    asm volatile("ld.shared::cluster.s64 %0, [%1];" : "=l"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ int ld_cl_s32(uint32_t a) {
    int v;
    asm volatile("ld.shared::cluster.s32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ void st_cl_f32(uint32_t a, float v) {
    asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(a), "f"(v));
}

// packed FP32 pairs (f32x2 arithmetic, round to nearest like the scalar ops)
typedef unsigned long long f2;
__device__ __forceinline__ f2 pk(float a, float b) {
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void upk(f2 v, float& a, float& b) { asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v)); }
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) {
    f2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b) {
    f2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 sub2(f2 a, f2 b) {
    f2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 add2(f2 a, f2 b) {
    f2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// ---------------------------------------------------------------- accumulators
// A and R of a pass are summed in shared memory with atomic adds: FP32 (the
// order of the adds, and so the last bits of the sums, varies from run to
// run), or, in the deterministic build, 64-bit fixed point, whose integer adds
// do not depend on their order.  Fixed point: A_i has |A_i| <= 1/2 (sum_j
// P_ij <= 1 and |w d| <= 1/2), kept at 2^-61; R_i has |R_i| <= 0.33 (z - 1)
// < 2700 (|w^2 d| <= 0.33), kept at 2^-48; both stay below 2^62.  The layout
// (quantity k of row i at k zcap + i) is the same; a deterministic entry is
// 8 bytes.
constexpr float kFixA = 2305843009213693952.0f;   // 2^61
constexpr float kFixR = 281474976710656.0f;       // 2^48
// One block's view of the accumulators.  Whole sums (the FP32 build, and the
// deterministic build where they leave the block the warps asked for): every
// block holds all rows (quantity q of row i at q * stride + i, stride = zcap).
// Split sums (the deterministic build on a cluster of K > 1 blocks
// otherwise): block r holds rows [r slice, (r + 1) slice) only (quantity q
// of its local row l at q * stride + l), and an add to another block's row
// goes to that block's shared memory (a cluster-scope reduction), so that
// each block's 8-byte sums take 1 / K of the space.
struct AccRef {
    float* p;
    int stride;
    int slice;
    uint32_t rank, K;
};
__device__ __forceinline__ void red_cl_add_u64(uint32_t a, unsigned long long v) {
    asm volatile("red.shared::cluster.add.u64 [%0], %1;" ::"r"(a), "l"(v) : "memory");
}
template <bool DET>
__device__ __forceinline__ void acc_add(const AccRef& A, int q, int i, float v, bool isR) {
    if constexpr (DET) {
        const unsigned long long x = (unsigned long long)__float2ll_rn(v * (isR ? kFixR : kFixA));
        uint32_t owner = 0;
        if (A.K > 1)
            owner = (uint32_t)(i >= A.slice) + (A.K > 2 ? (uint32_t)(i >= 2 * A.slice) + (uint32_t)(i >= 3 * A.slice) : 0u);
        unsigned long long* a = reinterpret_cast<unsigned long long*>(A.p) + (q * A.stride + i - (int)owner * A.slice);
        if (owner == A.rank) atomicAdd(a, x);
        else red_cl_add_u64(map_rank(smem_u32(a), owner), x);
    } else {
        atomicAdd(A.p + q * A.stride + i, v);
    }
}

// ---------------------------------------------------------------- tile evaluation
// The shared map of a 2-D chunk is stored as column pairs, float4 k = (x_2k,
// x_2k+1, y_2k, y_2k+1), so that a lane reads the two columns of a step with
// one 16-byte load; a 3-D map is structure-of-arrays (coordinate k of row i
// at map[k * zcap + i]).
template <int OD>
__device__ __forceinline__ int map_idx(int zcap, int i, int k) {
    if constexpr (OD == 2) return ((i >> 1) << 2) | (k << 1) | (i & 1);
    else return k * zcap + i;
}
//
// One warp evaluates a whole 32 x 32 tile (rows of block a, columns
// of block b).  Lane L = 16 h + g owns rows 2g and 2g + 1 of a and the ring h
// of b's columns 16h..16h+15, met in the order (g + t) & 15, two columns per
// double step s (t = 2s, 2s + 1).  Per pair: w = 1 / (1 + |y_i - y_j|^2) and
// the terms p w (y_i - y_j) and w^2 (y_i - y_j) of A and R, plus w for Z.
//
// Off-diagonal tile (a != b): every unordered pair is evaluated once.  Its
// terms go to the lane's row sums and, with the opposite sign, to a column
// packet (the sums of the two columns of the double step).  After each double
// step the packets move two lanes down the ring (lane g receives from lane
// g + 2), so the packet of columns (c, c + 1) meets the 8 lanes g = c - 2s;
// at the end lane g holds column (g - 2)'s partial and column (g - 1)'s, and
// the two partials of a column (from lanes of either parity) are added.
// Diagonal tile (a == b): both (i, j) and (j, i) are stored, so the tile is
// evaluated row-wise only, every ordered pair once.
//
// Rows and columns at or beyond z are padding far from everything (see kPad):
// their pairs add nothing, and their own sums are never read.

__device__ __forceinline__ f2 shfl_f2(f2 v, int src) {
    float lo, hi;
    upk(v, lo, hi);
    lo = __shfl_sync(0xffffffffu, lo, src);
    hi = __shfl_sync(0xffffffffu, hi, src);
    return pk(lo, hi);
}
__device__ __forceinline__ float hsum2(f2 v) {
    float lo, hi;
    upk(v, lo, hi);
    return lo + hi;
}

// A lane's 32 P values: its float4 f = 0..7 (see packed_index), float4
// f * 32 + lane of the tile, so that each of the eight accesses of a warp
// touches 512 contiguous bytes.
__device__ __forceinline__ void tile_lane_values(const float* tile, int lane, float4 (&pv)[8]) {
    const float4* base = reinterpret_cast<const float4*>(tile) + lane;
#pragma unroll
    for (int s = 0; s < 8; ++s) pv[s] = base[s * kPT];
}
// Copy a stored tile from HBM into the warp's shared buffer: lane l copies its
// own eight float4 (the ones it reads back), lane 0 the trailer too.
__device__ __forceinline__ void tile_copy_async(uint32_t buf_a, const float* tile, int lane) {
    const float4* src = reinterpret_cast<const float4*>(tile) + lane;
#pragma unroll
    for (int s = 0; s < 8; ++s) cp_async16(buf_a + (uint32_t)(s * kPT + lane) * 16u, src + s * kPT);
    if (lane == 0) cp_async16(buf_a + (uint32_t)kPTileFloats * 4u, tile + kPTileFloats);
    cp_async_commit();
}

// Row sums of 2 rows kept by one lane of the pair (h, h ^ 1): lane h keeps row
// 2g + h and adds the other lane's partial of it.
__device__ __forceinline__ float keep_row(float mine0, float mine1, int h) {
    const float keep = h ? mine1 : mine0, give = h ? mine0 : mine1;
    return keep + __shfl_xor_sync(0xffffffffu, give, 16);
}

// Gradient sums of 2-D maps (packed f32x2 over the two columns of a step).
// Lane L = 8 q + g holds rows 4g .. 4g+3 of row block a (the map's column
// pairs 2g and 2g + 1) and meets the 8 columns of ring q of block b as the
// natural column pairs (g / 2 + s) & 3, s = 0..3, each read as one float4
// (x, x', y, y').  A warp keeps the row sums of its current row block across
// the tiles it takes in a row (the stored tiles come row block by row block,
// so consecutive tiles of a warp often share a) and adds them to acc when the
// row block changes or the pass ends (rows2_flush).
struct Rows2 {
    f2 OX[4], OY[4];                     // the lane's four rows, duplicated into both halves
    f2 AX[4], AY[4], RX[4], RY[4];       // their partial sums over the columns met so far
};

__device__ __forceinline__ void rows2_begin(Rows2& R, const float* map, int a, int lane) {
    const float4* mp = reinterpret_cast<const float4*>(map);
    const int g = lane & 7;
    const float4 o0 = mp[a * 16 + 2 * g], o1 = mp[a * 16 + 2 * g + 1];
    R.OX[0] = pk(o0.x, o0.x); R.OX[1] = pk(o0.y, o0.y); R.OX[2] = pk(o1.x, o1.x); R.OX[3] = pk(o1.y, o1.y);
    R.OY[0] = pk(o0.z, o0.z); R.OY[1] = pk(o0.w, o0.w); R.OY[2] = pk(o1.z, o1.z); R.OY[3] = pk(o1.w, o1.w);
#pragma unroll
    for (int r = 0; r < 4; ++r) R.AX[r] = R.AY[r] = R.RX[r] = R.RY[r] = 0ull;
}

// The row sums of the four rings are reduced over lanes g, g + 8, g + 16,
// g + 24, each keeping one row, and added to acc.
template <bool DET>
__device__ __forceinline__ void rows2_flush(const Rows2& R, int a, int lane, const AccRef& acc) {
    const int g = lane & 7, q = lane >> 3;
    float v[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        v[r][0] = hsum2(R.AX[r]);
        v[r][1] = hsum2(R.AY[r]);
        v[r][2] = hsum2(R.RX[r]);
        v[r][3] = hsum2(R.RY[r]);
    }
    // ring q keeps row 4g + 2 (q >> 1) + (q & 1) of the four rings' sums
    const bool hi = q >= 2, odd = q & 1;
    float w2[2][4];
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const float keep = hi ? v[2 + h][k] : v[h][k];
            const float give = hi ? v[h][k] : v[2 + h][k];
            w2[h][k] = keep + __shfl_xor_sync(0xffffffffu, give, 16);
        }
    const int row = a * kPT + 4 * g + (hi ? 2 : 0) + (odd ? 1 : 0);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float keep = odd ? w2[1][k] : w2[0][k];
        const float give = odd ? w2[0][k] : w2[1][k];
        acc_add<DET>(acc, k, row, keep + __shfl_xor_sync(0xffffffffu, give, 8), k >= 2);
    }
}

// One tile (rows of R's block, columns of block b).  Off-diagonal tile: the
// column packet of a step (the sums of its two columns over the lane's four
// rows) moves two lanes down the ring after each step (lane g receives from
// lane g + 2), so it meets the four lanes of one parity; lanes g and g ^ 1
// end with the two partial packets of pair (g / 2 - 1) & 3, each keeps one
// column and adds it to acc.  Diagonal tile: both orders are stored, rows
// only.  Returns the lane's sum of w (both orders of each pair of an
// off-diagonal tile).  After the first step it starts the copy of the
// warp's next tile nsrc (if any) into the warp's buffer at buf_a.
template <bool SYM, bool DET>
__device__ __forceinline__ float tile_grad_2d(Rows2& R, const float* map, int zcap, int b, int lane,
                                              const float4 (&pv)[8], const AccRef& acc, const float* nsrc, uint32_t buf_a) {
    const float4* mp = reinterpret_cast<const float4*>(map);
    const int g = lane & 7, q = lane >> 3, u = g >> 1;
    const f2 ONE = pk(1.f, 1.f);
    f2 Z = 0;
    f2 CAX = 0, CAY = 0, CRX = 0, CRY = 0;   // column packet (SYM)
    const int nxt = (lane & 24) | ((g + 2) & 7);
    const float4* cbase = mp + b * 16 + 4 * q;
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        const float4 cv = cbase[(u + s) & 3];
        const f2 XC = pk(cv.x, cv.y), YC = pk(cv.z, cv.w);
        const f2 P[4] = {pk(pv[2 * s].x, pv[2 * s].y), pk(pv[2 * s].z, pv[2 * s].w),
                         pk(pv[2 * s + 1].x, pv[2 * s + 1].y), pk(pv[2 * s + 1].z, pv[2 * s + 1].w)};
        f2 DX[4], DY[4], W[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            DX[r] = sub2(R.OX[r], XC);   // own - other
            DY[r] = sub2(R.OY[r], YC);
            f2 Q = fma2(DX[r], DX[r], ONE);
            Q = fma2(DY[r], DY[r], Q);
            float q0, q1;
            upk(Q, q0, q1);
            W[r] = pk(hw_rcp(q0), hw_rcp(q1));
        }
        Z = add2(Z, add2(add2(W[0], W[1]), add2(W[2], W[3])));
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const f2 PW = mul2(P[r], W[r]), WW = mul2(W[r], W[r]);
            R.AX[r] = fma2(PW, DX[r], R.AX[r]);
            R.AY[r] = fma2(PW, DY[r], R.AY[r]);
            R.RX[r] = fma2(WW, DX[r], R.RX[r]);
            R.RY[r] = fma2(WW, DY[r], R.RY[r]);
            if constexpr (SYM) {
                CAX = fma2(PW, DX[r], CAX);
                CAY = fma2(PW, DY[r], CAY);
                CRX = fma2(WW, DX[r], CRX);
                CRY = fma2(WW, DY[r], CRY);
            }
        }
        if constexpr (SYM) {
            if (s < 3) {
                CAX = shfl_f2(CAX, nxt);
                CAY = shfl_f2(CAY, nxt);
                CRX = shfl_f2(CRX, nxt);
                CRY = shfl_f2(CRY, nxt);
            }
        }
        if (s == 0 && nsrc) {
            // the next tile's copy into the buffer this tile came from: every
            // read of it has returned (the registers are used here)
            asm volatile("" ::"f"(pv[0].x), "f"(pv[1].x), "f"(pv[2].x), "f"(pv[3].x), "f"(pv[4].x), "f"(pv[5].x),
                         "f"(pv[6].x), "f"(pv[7].x)
                         : "memory");
            __syncwarp();
            tile_copy_async(buf_a, nsrc, lane);
        }
    }
    if constexpr (SYM) {
        const int oddg = g & 1;
        const int col = b * kPT + 8 * q + 2 * ((u + 3) & 3) + oddg;
        float lo, hv;
        upk(CAX, lo, hv);
        acc_add<DET>(acc, 0, col, -((oddg ? hv : lo) + __shfl_xor_sync(0xffffffffu, oddg ? lo : hv, 1)), false);
        upk(CAY, lo, hv);
        acc_add<DET>(acc, 1, col, -((oddg ? hv : lo) + __shfl_xor_sync(0xffffffffu, oddg ? lo : hv, 1)), false);
        upk(CRX, lo, hv);
        acc_add<DET>(acc, 2, col, -((oddg ? hv : lo) + __shfl_xor_sync(0xffffffffu, oddg ? lo : hv, 1)), true);
        upk(CRY, lo, hv);
        acc_add<DET>(acc, 3, col, -((oddg ? hv : lo) + __shfl_xor_sync(0xffffffffu, oddg ? lo : hv, 1)), true);
        return 2.0f * hsum2(Z);
    }
    return hsum2(Z);
}

// Same sums for 3-D maps (scalar arithmetic, same lane order and packets).
template <bool SYM, bool DET>
__device__ __forceinline__ float tile_grad_3d(const float* map, int zcap, int a, int b, int lane,
                                              const float4 (&pv)[8], const AccRef& acc) {
    const int g = lane & 15, h = lane >> 4;
    const int ra = a * kPT + 2 * g, cb = b * kPT + 16 * h;
    const float* pf = reinterpret_cast<const float*>(pv);
    float o[2][3], ra_[2][3], rr_[2][3], ca[2][3], cr[2][3];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            o[r][k] = map[k * zcap + ra + r];
            ra_[r][k] = 0.f;
            rr_[r][k] = 0.f;
            ca[r][k] = 0.f;
            cr[r][k] = 0.f;
        }
    float z = 0.f;
    const int nxt = (lane & 16) | ((g + 2) & 15);
#pragma unroll
    for (int s = 0; s < 8; ++s) {
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int cc = cb + ((g + 2 * s + e) & 15);
            float xc[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) xc[k] = map[k * zcap + cc];
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                float d[3], q = 1.0f;
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    d[k] = o[r][k] - xc[k];
                    q = fmaf(d[k], d[k], q);
                }
                const float w = hw_rcp(q);
                z += w;
                const float pw = pf[4 * s + 2 * r + e] * w, ww = w * w;
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    ra_[r][k] = fmaf(pw, d[k], ra_[r][k]);
                    rr_[r][k] = fmaf(ww, d[k], rr_[r][k]);
                    if constexpr (SYM) {
                        ca[e][k] = fmaf(pw, d[k], ca[e][k]);
                        cr[e][k] = fmaf(ww, d[k], cr[e][k]);
                    }
                }
            }
        }
        if constexpr (SYM) {
            if (s < 7) {
#pragma unroll
                for (int e = 0; e < 2; ++e)
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        ca[e][k] = __shfl_sync(0xffffffffu, ca[e][k], nxt);
                        cr[e][k] = __shfl_sync(0xffffffffu, cr[e][k], nxt);
                    }
            }
        }
    }
    const int row = ra + h;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        acc_add<DET>(acc, k, row, keep_row(ra_[0][k], ra_[1][k], h), false);
        acc_add<DET>(acc, 3 + k, row, keep_row(rr_[0][k], rr_[1][k], h), true);
    }
    if constexpr (SYM) {
        const int prv = (lane & 16) | ((g + 15) & 15);
        const int col = cb + ((g + 14) & 15);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            acc_add<DET>(acc, k, col, -(ca[0][k] + __shfl_sync(0xffffffffu, ca[1][k], prv)), false);
            acc_add<DET>(acc, 3 + k, col, -(cr[0][k] + __shfl_sync(0xffffffffu, cr[1][k], prv)), true);
        }
        return 2.0f * z;
    }
    return z;
}

// Cost sums of a lane's 32 pairs: sum p ln p, sum p ln w, sum p, sum w (Eq. 5,
// Eq. 9), doubled for an off-diagonal tile (each pair stands for both orders).
// 2-D maps: the ring-8 lane layout of tile_grad_2d.
template <bool SYM>
__device__ __forceinline__ void tile_cost_2d(const float* map, int a, int b, int lane, const float4 (&pv)[8],
                                             float (&c)[4]) {
    const float4* mp = reinterpret_cast<const float4*>(map);
    const int g = lane & 7, q = lane >> 3, u = g >> 1;
    const float4 o0 = mp[a * 16 + 2 * g], o1 = mp[a * 16 + 2 * g + 1];
    const float ox[4] = {o0.x, o0.y, o1.x, o1.y}, oy[4] = {o0.z, o0.w, o1.z, o1.w};
    const float* pf = reinterpret_cast<const float*>(pv);
    c[0] = c[1] = c[2] = c[3] = 0.f;
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        const float4 cv = mp[b * 16 + 4 * q + ((u + s) & 3)];
        const float cx[2] = {cv.x, cv.y}, cy[2] = {cv.z, cv.w};
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const float dx = ox[r] - cx[e], dy = oy[r] - cy[e];
                const float qv = fmaf(dy, dy, fmaf(dx, dx, 1.0f));
                c[3] += hw_rcp(qv);
                const float p = pf[4 * (2 * s + (r >> 1)) + ((r & 1) << 1) + e];
                if (p >= FLT_MIN) {
                    c[0] += p * (hw_lg2(p) * kLn2f);
                    c[1] -= p * (hw_lg2(qv) * kLn2f);
                    c[2] += p;
                }
            }
    }
    if constexpr (SYM) {
#pragma unroll
        for (int k = 0; k < 4; ++k) c[k] *= 2.0f;
    }
}

// 3-D maps: the ring-16 lane layout of tile_grad_3d.
template <int OD, bool SYM>
__device__ __forceinline__ void tile_cost(const float* map, int zcap, int a, int b, int lane, const float4 (&pv)[8],
                                          float (&c)[4]) {
    const int g = lane & 15, h = lane >> 4;
    const int ra = a * kPT + 2 * g, cb = b * kPT + 16 * h;
    const float* pf = reinterpret_cast<const float*>(pv);
    c[0] = c[1] = c[2] = c[3] = 0.f;
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        float o[OD];
#pragma unroll
        for (int k = 0; k < OD; ++k) o[k] = map[k * zcap + ra + r];
#pragma unroll
        for (int t = 0; t < 16; ++t) {
            const int cc = cb + ((g + t) & 15);
            float q = 1.0f;
#pragma unroll
            for (int k = 0; k < OD; ++k) {
                const float d = o[k] - map[k * zcap + cc];
                q = fmaf(d, d, q);
            }
            c[3] += hw_rcp(q);
            const float p = pf[4 * (t >> 1) + 2 * r + (t & 1)];
            if (p >= FLT_MIN) {
                c[0] += p * (hw_lg2(p) * kLn2f);
                c[1] -= p * (hw_lg2(q) * kLn2f);
                c[2] += p;
            }
        }
    }
    if constexpr (SYM) {
#pragma unroll
        for (int k = 0; k < 4; ++k) c[k] *= 2.0f;
    }
}

// Stored tiles of one block of the cluster: a contiguous share of the
// chunk's stored tiles (stored row block by row block), so that a warp's
// consecutive tiles share their row block as often as possible; the K shares
// differ in length by at most one tile.
struct Stream {
    int first, nq;   // this block's tiles of the chunk: stored tiles first .. first + nq - 1, per pass
    __device__ Stream(int nb, uint32_t rank, uint32_t K) {
        const long long total = (long long)nb * (nb + 1) / 2;
        first = (int)(total * rank / K);
        nq = (int)(total * (rank + 1) / K) - first;
    }
};

// Compensated FP32 running sum (per lane; combined in FP64 at the end of a pass).
struct KSum {
    float s, c;
    __device__ __forceinline__ void clear() { s = 0.f; c = 0.f; }
    __device__ __forceinline__ void add(float v) {
        const float y = v - c, t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

// s + v with the rounding error carried in c (error-free two-sum)
__device__ __forceinline__ void two_sum_add(float& s, float& c, float v, float cv) {
    const float t = s + v;
    const float bb = t - s;
    const float e = (s - (t - bb)) + (v - bb);
    s = t;
    c = c + cv + e;
}
// Sum over the warp of the lanes' compensated sums, exact to the FP32 sum of
// the rounding errors (error-free two-sums on the shuffles; FP64 arithmetic,
// slow on this GPU, only for lane 0's final conversion); lane 0 holds it.
__device__ __forceinline__ double warp_sum_ksum(const KSum& k) {
    float hi = k.s, lo = -k.c;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float h2 = __shfl_xor_sync(0xffffffffu, hi, o), l2 = __shfl_xor_sync(0xffffffffu, lo, o);
        two_sum_add(hi, lo, h2, l2);
    }
    return (double)hi + (double)lo;
}

// A warp's n_w tiles of one pass: tile j is stored at P2w + j * step (the
// block's tile w + j W).  The warp owns one shared buffer: on entry it holds
// (or is receiving) tile 0; for each tile the warp waits for its copy, reads
// it into registers, starts the copy of the next tile into the buffer (after
// the pass's last tile, the next pass's first when `more`; nothing after the
// chunk's last), then evaluates (COST: the cost sums instead of the gradient
// sums).  The copy of the next tile thus has a whole tile's arithmetic to
// land (an L2 prefetch of the tile after that measured slower: its
// instructions cost more than the latency they hide).  In a 2-D gradient
// pass the copy starts after the tile's first step, by when the warp's
// reads of the buffer have long returned (measured 1.5% faster than
// waiting for them before the first step).
template <int OD, bool COST, bool DET>
__device__ __forceinline__ void consume_pass(const float* P2b, int w0, int n_w, int next0, int nb, const float* buf,
                                             const float* map, int zcap, const AccRef& acc, int lane, KSum (&part)[4]) {
    // w of the pair (i, i), which a diagonal tile's row-wise pass counts in
    // its lanes with h == g / 8 (rows 2g, 2g + 1 meet their own columns)
    // (ring-8 layout: lanes with q == g / 2 meet their own four rows;
    // ring-16: lanes with h == g / 8 meet their own two rows)
    const float w_ii = hw_rcp(1.0f);
    const bool diag_lane = OD == 2 ? (lane >> 3) == ((lane & 7) >> 1) : (lane >> 4) == ((lane & 15) >> 3);
    constexpr float kDiagPairs = OD == 2 ? 4.0f : 2.0f;
    const uint32_t buf_a = smem_u32(buf);
    Rows2 R;          // 2-D gradient pass: the row sums of row block cur_a
    int cur_a = -1;
    for (int j = 0; j < n_w; ++j) {
        cp_async_wait_all();   // this lane's part of the tile (and lane 0's trailer) ...
        __syncwarp();          // ... and every lane's, visible to the warp
        const int2 ab = *reinterpret_cast<const int2*>(buf + kPTileFloats);
        float4 pv[8];
        tile_lane_values(buf, lane, pv);
        const int qn = j + 1 < n_w ? w0 + j + 1 : next0;
        const float* nsrc = qn >= 0 ? P2b + (int64_t)qn * kPTileStride : nullptr;
        if (OD != 2 || COST) {
            // the reads have returned (their registers are used here) before the
            // next copy may overwrite the buffer
            asm volatile("" ::"f"(pv[0].x), "f"(pv[1].x), "f"(pv[2].x), "f"(pv[3].x), "f"(pv[4].x), "f"(pv[5].x),
                         "f"(pv[6].x), "f"(pv[7].x), "r"(ab.x), "r"(ab.y)
                         : "memory");
            __syncwarp();
            if (nsrc) tile_copy_async(buf_a, nsrc, lane);
        } else {
            asm volatile("" ::"r"(ab.x), "r"(ab.y) : "memory");   // (the trailer's read has returned)
        }
        // the trailer is written by the joint-P kernel; clamp it anyway so
        // that no shared-memory index can leave the chunk's rows
        const int a = (int)min((unsigned)ab.x, (unsigned)(nb - 1)), b = (int)min((unsigned)ab.y, (unsigned)(nb - 1));
        const bool diag = a == b;
        const float drop = diag && diag_lane ? kDiagPairs * w_ii : 0.0f;
        if constexpr (!COST) {
            float zl;
            if constexpr (OD == 2) {
                if (a != cur_a) {   // warp-uniform: a new row block
                    if (cur_a >= 0) rows2_flush<DET>(R, cur_a, lane, acc);
                    rows2_begin(R, map, a, lane);
                    cur_a = a;
                }
                zl = diag ? tile_grad_2d<false, DET>(R, map, zcap, b, lane, pv, acc, nsrc, buf_a)
                          : tile_grad_2d<true, DET>(R, map, zcap, b, lane, pv, acc, nsrc, buf_a);
            } else {
                zl = diag ? tile_grad_3d<false, DET>(map, zcap, a, b, lane, pv, acc)
                          : tile_grad_3d<true, DET>(map, zcap, a, b, lane, pv, acc);
            }
            part[0].add(zl - drop);
        } else {
            float cs[4];
            if constexpr (OD == 2) {
                if (diag) tile_cost_2d<false>(map, a, b, lane, pv, cs);
                else tile_cost_2d<true>(map, a, b, lane, pv, cs);
            } else {
                if (diag) tile_cost<OD, false>(map, zcap, a, b, lane, pv, cs);
                else tile_cost<OD, true>(map, zcap, a, b, lane, pv, cs);
            }
            part[0].add(cs[3] - drop);
            part[1].add(cs[0]);
            part[2].add(cs[1]);
            part[3].add(cs[2]);
        }
    }
    if constexpr (OD == 2 && !COST) {
        if (cur_a >= 0) rows2_flush<DET>(R, cur_a, lane, acc);
    }
}

// Compiled for at most MAXT threads.  2-D maps: 512 (16 warps) or 384 (12),
// both 128 registers per thread.  3-D maps: 672 (21 warps, 80 registers) or
// 544 (17, 96 registers).  Registers are granted per 4 warps, so 21 warps
// get 80, 17 to 20 warps 96 and 16 or fewer 128.
template <int OD, int MAXT, bool DET>
__global__ void __launch_bounds__(MAXT, 1) iterate_kernel(IterArgs A) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nthreads = blockDim.x;
    const int W = nthreads >> 5;                    // warps, each evaluating tiles
    const int zcap = A.zcap;

    // one tile buffer per warp (4112 bytes: P and trailer), then the map and
    // the accumulators
    float* wbuf = reinterpret_cast<float*>(smem_raw) + (size_t)warp * kPTileStride;
    float* map = reinterpret_cast<float*>(smem_raw) + (size_t)W * kPTileStride;   // OD arrays of zcap floats
    float* acc = map + (size_t)OD * zcap;                                         // 2*OD arrays: A_0.., R_0..

    __shared__ double s_red[32][4];
    __shared__ double s_part[4];                    // this block's Z (and cost) partial sums
    __shared__ int s_item;
    __shared__ float s_mn[32], s_mx[32];
    __shared__ float s_eta;
    __shared__ float s_invZ;                        // 1 / Z of the pass
    __shared__ int s_cut[2][kMaxWarps + 1];        // warp pieces of the block's share: passes 0-1, passes 2+
    __shared__ long long s_cyc[kMaxWarps];          // each warp's cycles in the chunk's first pass

    const uint32_t K = cl_size(), rank = cl_rank();
    for (;;) {
        if (rank == 0 && tid == 0) s_item = atomicAdd(A.queue, 1);
        sync_owner(K);
        const int item = (K > 1) ? ld_cl_s32(map_rank(smem_u32(&s_item), 0)) : s_item;
        sync_owner(K);
        if (item >= A.L.n_chunks) break;

        const int c = A.L.order[item];
        const int64_t off = A.L.off[c];
        const int z = (int)(A.L.off[c + 1] - off);
        const int nb = (z + kPT - 1) / kPT;
        const int zr = nb * kPT;
        const Stream S(nb, rank, K);
        // rows updated by this block; the deterministic build on a cluster
        // splits the accumulators the same way (over the zr padded rows, which
        // all receive sums), each block holding its own rows' sums
        const bool split = DET && K > 1 && A.acc_rows < zcap;   // chosen by the launcher
        const int slice = split ? (zr + (int)K - 1) / (int)K : (z + (int)K - 1) / (int)K;
        const int ulo = (int)rank * slice, uhi = min(z, ulo + slice);
        // (whole sums: every add is local, owner 0 of a one-block view)
        const AccRef accr{acc, split ? A.acc_rows : zcap, slice, split ? rank : 0u, split ? K : 1u};
        const int npass = A.iters + (A.cost_pass ? 1 : 0);

        // this warp's tiles of the chunk: a contiguous piece of the block's
        // share (so that its consecutive tiles share their row block: its row
        // sums are added to the accumulators once per row block), equal
        // pieces in the first two passes and, from the third, pieces sized to
        // each warp's measured rate in the first (the warps of a block do not
        // run at quite the same speed, and a pass waits for the slowest; the
        // deterministic build keeps equal pieces, whose FP32 partial sums do
        // not depend on timing); the copy of the first tile starts before the
        // map is even loaded
        const float* P2b = A.P2 + (A.ptile_off[c] + S.first) * kPTileStride;
        if (tid <= W) s_cut[0][tid] = s_cut[1][tid] = (int)((long long)S.nq * tid / W);
        {
            const int w0 = (int)((long long)S.nq * warp / W);
            if ((int)((long long)S.nq * (warp + 1) / W) > w0)
                tile_copy_async(smem_u32(wbuf), P2b + (int64_t)w0 * kPTileStride, lane);
        }

        for (int i = tid; i < zr; i += nthreads) {
#pragma unroll
            for (int k = 0; k < OD; ++k) map[map_idx<OD>(zcap, i, k)] = i < z ? A.Yc[(off + i) * OD + k] : kPad * (float)(i - z + 1);
        }
        for (int i = tid; i < (DET ? 4 : 2) * OD * accr.stride; i += nthreads) acc[i] = 0.f;
        __syncthreads();
        if (split) cl_barrier();   // every block's sums are zero before any block adds to them

        for (int it = 0; it < npass; ++it) {
            const bool cost = it == A.iters;
            if (!cost && A.opt.lr_mode == PTSNE_LR_PAPER) {
                float mn = FLT_MAX, mx = -FLT_MAX;
                for (int i = tid; i < z; i += nthreads)
#pragma unroll
                    for (int k = 0; k < OD; ++k) {
                        mn = fminf(mn, map[map_idx<OD>(zcap, i, k)]);
                        mx = fmaxf(mx, map[map_idx<OD>(zcap, i, k)]);
                    }
                mn = warp_min(mn);
                mx = warp_max(mx);
                if (lane == 0) { s_mn[warp] = mn; s_mx[warp] = mx; }
                __syncthreads();
                if (tid == 0) {
                    float a = FLT_MAX, b = -FLT_MAX;
                    for (int w = 0; w < W; ++w) { a = fminf(a, s_mn[w]); b = fmaxf(b, s_mx[w]); }
                    s_eta = step_eta(A.opt, z, a, b);
                }
            }

            KSum part[4];                              // Z, sum p ln p, sum p ln w, sum p
#pragma unroll
            for (int k = 0; k < 4; ++k) part[k].clear();
            const int* cut = s_cut[it >= 2 ? 1 : 0];
            const int* cut_n = s_cut[it + 1 >= 2 ? 1 : 0];
            const int w0 = cut[warp], n_w = cut[warp + 1] - w0;
            // the next pass's first tile of this warp (none after the chunk's
            // last pass, or if its next piece is empty)
            const int next0 = it + 1 < npass && cut_n[warp + 1] > cut_n[warp] ? cut_n[warp] : -1;
            const long long t_pass = clock64();
            if (!cost) consume_pass<OD, false, DET>(P2b, w0, n_w, next0, nb, wbuf, map, zcap, accr, lane, part);
            else consume_pass<OD, true, DET>(P2b, w0, n_w, next0, nb, wbuf, map, zcap, accr, lane, part);
            if (it == 0 && lane == 0) s_cyc[warp] = clock64() - t_pass;
            // block partials (fixed order), then the cluster total; a gradient pass
            // has only Z (the cost sums are zero there)
            const int nsum = cost ? 4 : 1;
            for (int k = 0; k < nsum; ++k) {
                const double v = warp_sum_ksum(part[k]);
                if (lane == 0) s_red[warp][k] = v;
            }
            __syncthreads();
            if (!DET && it == 0 && tid == 0 && S.nq >= 16 * W) {   // (deterministic: the pieces stay fixed)
                // pieces from the third pass on: proportional to each warp's
                // rate (tiles per cycle) in the first pass
                float tot = 0.f;
                for (int w = 0; w < W; ++w) tot += (float)(s_cut[0][w + 1] - s_cut[0][w]) / (float)max(s_cyc[w], 1ll);
                float acc_r = 0.f;
                for (int w = 0; w < W; ++w) {
                    const float rate = (float)(s_cut[0][w + 1] - s_cut[0][w]) / (float)max(s_cyc[w], 1ll);
                    s_cut[1][w] = min(S.nq, (int)((float)S.nq * (acc_r / tot) + 0.5f));
                    acc_r += rate;
                }
                s_cut[1][W] = S.nq;
            }
            if (tid < nsum) {
                double v = 0.0;
                for (int w = 0; w < W; ++w) v += s_red[w][tid];
                s_part[tid] = v;
            }
            sync_owner(K);
            // the cluster totals (FP64, in rank order), by one thread: FP64
            // arithmetic is slow on this GPU, so the block's other threads
            // take 1 / Z from shared memory
            if (tid == 0) {
                double tot[4] = {0.0, 0.0, 0.0, 0.0};
                for (uint32_t rr = 0; rr < K; ++rr)
                    for (int k = 0; k < nsum; ++k)
                        tot[k] += K > 1 ? ld_cl_f64(map_rank(smem_u32(&s_part[k]), rr)) : s_part[k];
                if (cost) {
                    if (rank == 0) {
                        const double lnZ = log(tot[0]);
                        A.cost_chunk[2 * c] = tot[1] - tot[2] + tot[3] * lnZ;
                        A.cost_chunk[2 * c + 1] = (-tot[2] + tot[3] * lnZ) / (log((double)z) + log((double)(z - 1)));
                    }
                } else {
                    if (rank == 0 && A.Zc) A.Zc[c] = tot[0];
                    s_invZ = (float)(1.0 / tot[0]);
                }
            }
            __syncthreads();
            if (!cost) {
                const float invZ = s_invZ;
                const float eta = A.opt.lr_mode == PTSNE_LR_PAPER ? s_eta : A.opt.lr;
                // each thread's rows: every load of a row (the accumulators of
                // the cluster's blocks, the velocity and gains in HBM) is issued
                // before any of its arithmetic (two rows at a time measured
                // slower: the registers they take spill elsewhere)
                for (int i = ulo + tid; i < uhi; i += nthreads) {
                    const int64_t gi = (off + i) * OD;
                    float Av[OD], Rv[OD], y[OD], vel[OD], gn[OD];
#pragma unroll
                    for (int k = 0; k < OD; ++k) {
                        y[k] = map[map_idx<OD>(zcap, i, k)];
                        vel[k] = A.vel[gi + k];
                        gn[k] = A.gains[gi + k];
                        Av[k] = 0.f;
                        Rv[k] = 0.f;
                    }
                    if constexpr (DET) {   // integer sums (over the cluster), then to float
                        long long* acc64 = reinterpret_cast<long long*>(acc);
                        long long sa[OD], sr[OD];
#pragma unroll
                        for (int k = 0; k < OD; ++k) sa[k] = sr[k] = 0;
                        if (split) {   // this block holds the row's sums: read and clear them
                            const int l = i - ulo, st = accr.stride;
#pragma unroll
                            for (int k = 0; k < OD; ++k) {
                                sa[k] = acc64[k * st + l];
                                sr[k] = acc64[(OD + k) * st + l];
                                acc64[k * st + l] = 0;
                                acc64[(OD + k) * st + l] = 0;
                            }
                        }
                        for (uint32_t rr = 0; rr < (split ? 0u : K); ++rr) {
#pragma unroll
                            for (int k = 0; k < OD; ++k) {
                                if (K > 1) {
                                    sa[k] += ld_cl_s64(map_rank(smem_u32(acc64 + k * zcap + i), rr));
                                    sr[k] += ld_cl_s64(map_rank(smem_u32(acc64 + (OD + k) * zcap + i), rr));
                                } else {
                                    sa[k] += acc64[k * zcap + i];
                                    sr[k] += acc64[(OD + k) * zcap + i];
                                }
                            }
                        }
#pragma unroll
                        for (int k = 0; k < OD; ++k) {
                            Av[k] = (float)((double)sa[k] * (1.0 / (double)kFixA));
                            Rv[k] = (float)((double)sr[k] * (1.0 / (double)kFixR));
                        }
                    } else {
                        for (uint32_t rr = 0; rr < K; ++rr) {
#pragma unroll
                            for (int k = 0; k < OD; ++k) {
                                if (K > 1) {
                                    Av[k] += ld_cl_f32(map_rank(smem_u32(acc + k * zcap + i), rr));
                                    Rv[k] += ld_cl_f32(map_rank(smem_u32(acc + (OD + k) * zcap + i), rr));
                                } else {
                                    Av[k] += acc[k * zcap + i];
                                    Rv[k] += acc[(OD + k) * zcap + i];
                                }
                            }
                        }
                    }
                    update_point<OD>(y, vel, gn, Av, Rv, invZ, eta, A.opt, A.gradp ? A.gradp + gi : nullptr);
#pragma unroll
                    for (int k = 0; k < OD; ++k) {
                        A.vel[gi + k] = vel[k];
                        if (A.opt.use_gains) A.gains[gi + k] = gn[k];
                    }
                    for (uint32_t rr = 0; rr < K; ++rr)
#pragma unroll
                        for (int k = 0; k < OD; ++k) {
                            if (K > 1) st_cl_f32(map_rank(smem_u32(map + map_idx<OD>(zcap, i, k)), rr), y[k]);
                            else map[map_idx<OD>(zcap, i, k)] = y[k];
                        }
                }
            }
            if (split && !cost) {
                // the rest of this block's sums (padded rows, or a block with
                // no rows of this chunk): clear before the barrier below, after
                // which the other blocks add the next pass's sums
                long long* acc64 = reinterpret_cast<long long*>(acc);
                const int l0 = max(0, uhi - ulo), st = accr.stride;
                for (int l = l0 + tid; l < st; l += nthreads)
#pragma unroll
                    for (int q = 0; q < 2 * OD; ++q) acc64[q * st + l] = 0;
            }
            sync_owner(K);   // new map everywhere; remote reads of acc are done
            if (!split) {
                // 2 OD zcap entries of 4 (8 if DET) bytes, zcap a multiple of 32
                for (int i = tid; i < (DET ? 2 : 1) * OD * zcap / 2; i += nthreads)
                    reinterpret_cast<float4*>(acc)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
            __syncthreads();
        }
        for (int i = ulo + tid; i < uhi; i += nthreads)
#pragma unroll
            for (int k = 0; k < OD; ++k) A.Yc[(off + i) * OD + k] = map[map_idx<OD>(zcap, i, k)];
        __syncthreads();
    }
}

// ---------------------------------------------------------------- launchers

// Rows of one block's accumulators: all zcap, or, in the deterministic build
// on a cluster of K > 1 blocks, the block's own share (rounded up to 32).
int iterate_acc_rows(int64_t zmax, bool det, int K) {
    const int zcap = (int)((zmax + kPT - 1) / kPT * kPT);
    if (!det || K <= 1) return zcap;
    return ((zcap + K - 1) / K + kPT - 1) / kPT * kPT;
}

int iterate_smem_bytes(int od, int64_t zmax, int warps, bool det, int K) {
    const int zcap = (int)((zmax + kPT - 1) / kPT * kPT);
    // a tile buffer per warp, the map (a 2-D map as column pairs), A and R
    // (structure-of-arrays; 8-byte fixed point when deterministic)
    return warps * kPTileStride * 4 + zcap * od * 4 + iterate_acc_rows(zmax, det, K) * 2 * od * (det ? 8 : 4);
}

// Warps (at most `want`) whose tile buffers fit beside the map and the
// accumulators in 227 KB of shared memory; 0 if not even one fits.
int iterate_warps(int od, int64_t zmax, int want, bool det, int K) {
    int w = want;
    while (w > 0 && iterate_smem_bytes(od, zmax, w, det, K) > 227 * 1024 - kStaticSmem) --w;
    return w;
}

cudaError_t launch_iterate(const ptsne_ctx* c, int iters, int cost_pass, float* gradp, double* Zc, double* cost_chunk,
                           cudaStream_t s) {
    if (iters <= 0 && !cost_pass) return cudaSuccess;
    const int K = c->tune.cluster;
    if (c->tune.group != 1) return cudaErrorInvalidValue;
    int Wc = c->tune.consumer_warps;   // warps per block, each evaluating tiles
    // the 2-D evaluation (four rows per lane) needs 128 registers per thread,
    // which a block of at most 16 warps gets; 3-D maps run at most 21 warps;
    // very large chunks leave room for fewer tile buffers
    if (c->p.out_dim == 2 && Wc > 16) Wc = 16;
    if (c->p.out_dim == 3 && Wc > 21) Wc = 21;
    const bool det = c->deterministic;
    // deterministic sums: whole in every block, unless that leaves fewer
    // warps than asked for and the cluster can split them
    const int Wwhole = iterate_warps(c->p.out_dim, c->zmax, Wc, det, 1);
    const bool split = det && K > 1 && Wwhole < Wc;
    Wc = split ? iterate_warps(c->p.out_dim, c->zmax, Wc, det, K) : Wwhole;
    if (Wc < 1) return cudaErrorInvalidConfiguration;
    const size_t smem = (size_t)iterate_smem_bytes(c->p.out_dim, c->zmax, Wc, det, split ? K : 1);
    cudaError_t e = cudaMemsetAsync(c->queue, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    IterArgs a;
    a.P2 = c->P2;
    a.ptile_off = c->d_ptile_off;
    a.L = make_layout(c);
    a.Yc = c->Yc;
    a.vel = c->vel;
    a.gains = c->gains;
    a.gradp = gradp;
    a.Zc = Zc;
    a.cost_chunk = cost_chunk;
    a.iters = iters;
    a.cost_pass = cost_pass;
    a.opt = Optim{c->p.lr, c->p.momentum, c->p.lr_mode, c->p.use_gains};
    a.queue = c->queue;
    a.zcap = (int)((c->zmax + kPT - 1) / kPT * kPT);
    a.acc_rows = iterate_acc_rows(c->zmax, det, split ? K : 1);

    // the build for the fewest threads that hold the block: more registers per thread
    void (*kern)(IterArgs);
    if (c->p.out_dim == 2) {
        if (det) kern = Wc > 12 ? iterate_kernel<2, 512, true> : iterate_kernel<2, 384, true>;
        else kern = Wc > 12 ? iterate_kernel<2, 512, false> : iterate_kernel<2, 384, false>;
    } else {
        if (det) kern = Wc > 17 ? iterate_kernel<3, 672, true> : iterate_kernel<3, 544, true>;
        else kern = Wc > 17 ? iterate_kernel<3, 672, false> : iterate_kernel<3, 544, false>;
    }
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    cfg.blockDim = dim3((unsigned)(Wc * 32), 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    int clusters = sms / K;
    if (K > 1) {
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = (unsigned)K;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        cfg.gridDim = dim3((unsigned)K, 1, 1);
        int active = 0;
        if (cudaOccupancyMaxActiveClusters(&active, kern, &cfg) == cudaSuccess && active > 0) clusters = active;
        cudaGetLastError();
    }
    if (clusters > c->p.n_chunks) clusters = c->p.n_chunks;
    if (clusters < 1) clusters = 1;
    cfg.gridDim = dim3((unsigned)(clusters * K), 1, 1);
    e = cudaLaunchKernelEx(&cfg, kern, a);
    if (e != cudaSuccess) return e;
    return launched(c, 1);
}

}  // namespace ptsne
