// Octree construction on the device (Sec. 3.2.2 refinement, Sec. 3.2.3 2:1 balance) and
// the octant-to-octant neighbour table (o2o, Sec. 3.2.4).
//
// A tree is described by its sets of split boxes ("internal" boxes) per level, each a
// Morton-sorted array of keys (the Morton key of the box's anchor at full depth):
//   refinement  top down: the boxes of level l that the predicate splits, and their
//               children (8 per box in child order, so Morton-sorted again);
//   2:1 balance bottom up: a box of level k - 1 must be split if it contains a
//               same-size neighbour box (or itself) of a split box of level k; the
//               closure, applied from the finest level down, is the coarsest 26-balanced
//               refinement of the refined tree (Sec. 3.2.3);
//   leaves      the children of the split boxes of level l - 1 that are not split;
//   o2o         per leaf and direction, binary searches in the per-level leaf and split
//               sets.
// Sorting is a stable LSD radix sort of 64-bit keys written here; set operations are
// sort / unique / binary search.  Device memory of the build is allocated with
// cudaMalloc and freed before it returns.
#include <cuda_runtime.h>

#include <algorithm>
#include <memory>
#include <string>
#include <vector>

#include "ltsoct_internal.h"
#include "refine.h"

namespace ltsoct {

namespace {

constexpr uint64_t kNoKey = ~0ull;  // a candidate outside the domain (sorts last)

// ---------------------------------------------------------------------------
// device buffers of the build
// ---------------------------------------------------------------------------
template <typename T>
struct DBuf {
  T* p = nullptr;
  size_t n = 0;
  DBuf() = default;
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  ~DBuf() {
    if (p) cudaFree(p);
  }
  cudaError_t alloc(size_t count) {
    if (p) cudaFree(p);
    p = nullptr;
    n = count;
    return count ? cudaMalloc(&p, sizeof(T) * count) : cudaSuccess;
  }
};

#define OK(call)                             \
  do {                                       \
    const cudaError_t e_ = (call);           \
    if (e_ != cudaSuccess) return e_;        \
  } while (0)

int blocks_for(long long n, int threads) {
  const long long b = (n + threads - 1) / threads;
  return int(std::min<long long>(std::max<long long>(b, 1), 152 * 32));
}

// ---------------------------------------------------------------------------
// exclusive scan of unsigned counts (three phases: block scans, scan of the block
// totals, recursively, and their addition)
// ---------------------------------------------------------------------------
constexpr int kScanBlock = 1024;  // elements per block (512 threads, 2 each)

__global__ void __launch_bounds__(512) scan_blocks(const unsigned* in, unsigned* out, unsigned* sums, long long n) {
  __shared__ unsigned s[kScanBlock];
  const long long base = (long long)blockIdx.x * kScanBlock;
  for (int i = threadIdx.x; i < kScanBlock; i += blockDim.x) s[i] = base + i < n ? in[base + i] : 0u;
  __syncthreads();
  // Hillis-Steele inclusive scan over the block
  for (int off = 1; off < kScanBlock; off <<= 1) {
    unsigned v0 = 0, v1 = 0;
    const int i0 = threadIdx.x, i1 = threadIdx.x + 512;
    if (i0 >= off) v0 = s[i0 - off];
    if (i1 >= off) v1 = s[i1 - off];
    __syncthreads();
    s[i0] += v0;
    s[i1] += v1;
    __syncthreads();
  }
  for (int i = threadIdx.x; i < kScanBlock; i += blockDim.x)
    if (base + i < n) out[base + i] = i ? s[i - 1] : 0u;
  if (threadIdx.x == 0) sums[blockIdx.x] = s[kScanBlock - 1];
}

__global__ void scan_add(unsigned* out, const unsigned* sums, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] += sums[i / kScanBlock];
}

// out[i] = in[0] + ... + in[i-1]; *total (host) = the sum of all n
cudaError_t exclusive_scan(const unsigned* in, unsigned* out, long long n, unsigned* total, cudaStream_t s) {
  if (n <= 0) {
    *total = 0;
    return cudaSuccess;
  }
  const long long nb = (n + kScanBlock - 1) / kScanBlock;
  DBuf<unsigned> sums, sums_scan;
  OK(sums.alloc(nb));
  OK(sums_scan.alloc(nb));
  scan_blocks<<<unsigned(nb), 512, 0, s>>>(in, out, sums.p, n);
  OK(cudaGetLastError());
  unsigned last_in = 0, last_out = 0;
  if (nb > 1) {
    unsigned t = 0;
    OK(exclusive_scan(sums.p, sums_scan.p, nb, &t, s));
    scan_add<<<blocks_for(n, 256), 256, 0, s>>>(out, sums_scan.p, n);
    OK(cudaGetLastError());
  }
  OK(cudaMemcpyAsync(&last_in, in + n - 1, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  OK(cudaMemcpyAsync(&last_out, out + n - 1, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  OK(cudaStreamSynchronize(s));
  *total = last_in + last_out;
  return cudaSuccess;
}

// ---------------------------------------------------------------------------
// stable LSD radix sort of 64-bit keys on bits [lo, lo + bits), 8 bits per pass: per
// tile a digit histogram, a scan of the histograms in digit-major order, and a stable
// scatter (ranks within a warp from match masks, then across the warps of the tile)
// ---------------------------------------------------------------------------
constexpr int kSortThreads = 256, kSortChunks = 8, kSortTile = kSortThreads * kSortChunks;

__global__ void __launch_bounds__(kSortThreads) radix_hist(const uint64_t* keys, long long n, int shift,
                                                           unsigned* hist) {
  __shared__ unsigned h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const long long base = (long long)blockIdx.x * kSortTile;
  for (int k = 0; k < kSortChunks; ++k) {
    const long long i = base + k * kSortThreads + threadIdx.x;
    if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255u], 1u);
  }
  __syncthreads();
  hist[(long long)threadIdx.x * gridDim.x + blockIdx.x] = h[threadIdx.x];
}

__global__ void __launch_bounds__(kSortThreads) radix_scatter(const uint64_t* in, uint64_t* out, long long n, int shift,
                                                              const unsigned* offs) {
  __shared__ unsigned base[256];
  __shared__ unsigned wc[kSortThreads / 32][256];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  base[threadIdx.x] = offs[(long long)threadIdx.x * gridDim.x + blockIdx.x];
  const long long tile = (long long)blockIdx.x * kSortTile;
  for (int k = 0; k < kSortChunks; ++k) {
    for (int w = 0; w < kSortThreads / 32; ++w) wc[w][threadIdx.x] = 0;
    __syncthreads();
    const long long i = tile + k * kSortThreads + threadIdx.x;
    const bool valid = i < n;
    const uint64_t key = valid ? in[i] : 0ull;
    const unsigned d = valid ? unsigned((key >> shift) & 255u) : 256u;  // invalid lanes form their own group
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const unsigned rank = __popc(peers & ((1u << lane) - 1u));
    if (valid && rank == 0) wc[warp][d] = __popc(peers);
    __syncthreads();
    if (valid) {
      unsigned pre = 0;
      for (int w = 0; w < warp; ++w) pre += wc[w][d];
      out[base[d] + pre + rank] = key;
    }
    __syncthreads();
    unsigned add = 0;
    for (int w = 0; w < kSortThreads / 32; ++w) add += wc[w][threadIdx.x];
    base[threadIdx.x] += add;
    __syncthreads();
  }
}

// sorts keys[0, n) by bits [lo, lo + bits); tmp holds n keys
cudaError_t radix_sort(uint64_t* keys, uint64_t* tmp, long long n, int lo, int bits, cudaStream_t s) {
  if (n <= 1) return cudaSuccess;
  const long long tiles = (n + kSortTile - 1) / kSortTile;
  DBuf<unsigned> hist, offs;
  OK(hist.alloc(256 * tiles));
  OK(offs.alloc(256 * tiles));
  uint64_t* a = keys;
  uint64_t* b = tmp;
  for (int shift = lo; shift < lo + bits; shift += 8) {
    radix_hist<<<unsigned(tiles), kSortThreads, 0, s>>>(a, n, shift, hist.p);
    OK(cudaGetLastError());
    unsigned total = 0;
    OK(exclusive_scan(hist.p, offs.p, 256 * tiles, &total, s));
    radix_scatter<<<unsigned(tiles), kSortThreads, 0, s>>>(a, b, n, shift, offs.p);
    OK(cudaGetLastError());
    std::swap(a, b);
  }
  if (a != keys) OK(cudaMemcpyAsync(keys, a, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, s));
  return cudaSuccess;
}

// ---------------------------------------------------------------------------
// set operations on sorted key arrays
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool contains(const uint64_t* v, long long n, uint64_t key, long long* at = nullptr) {
  long long lo = 0, hi = n;
  while (lo < hi) {
    const long long mid = (lo + hi) >> 1;
    if (v[mid] < key)
      lo = mid + 1;
    else
      hi = mid;
  }
  if (at) *at = lo;
  return lo < n && v[lo] == key;
}

__global__ void unique_flags(const uint64_t* v, long long n, unsigned* flag) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    flag[i] = v[i] != kNoKey && (i == 0 || v[i] != v[i - 1]);
}

__global__ void compact(const uint64_t* in, const unsigned* flag, const unsigned* pos, long long n, uint64_t* out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    if (flag[i]) out[pos[i]] = in[i];
}

// keeps the entries of v with a nonzero flag (in order)
cudaError_t select(DBuf<uint64_t>& v, long long n, const unsigned* flag, long long* kept, cudaStream_t s) {
  DBuf<unsigned> pos;
  OK(pos.alloc(std::max<long long>(n, 1)));
  unsigned total = 0;
  OK(exclusive_scan(flag, pos.p, n, &total, s));
  DBuf<uint64_t> out;
  OK(out.alloc(std::max<unsigned>(total, 1u)));
  if (n) {
    compact<<<blocks_for(n, 256), 256, 0, s>>>(v.p, flag, pos.p, n, out.p);
    OK(cudaGetLastError());
  }
  OK(cudaStreamSynchronize(s));
  std::swap(v.p, out.p);
  std::swap(v.n, out.n);
  *kept = total;
  return cudaSuccess;
}

// sorts v[0, n), a level's keys (multiples of 8^(kDepth - level), or kNoKey), and drops
// duplicates and kNoKey
cudaError_t sort_unique(DBuf<uint64_t>& v, long long n, int level, long long* kept, cudaStream_t s) {
  if (n == 0) {
    *kept = 0;
    return cudaSuccess;
  }
  DBuf<uint64_t> tmp;
  OK(tmp.alloc(n));
  const int lo = 3 * (kDepth - level);
  OK(radix_sort(v.p, tmp.p, n, lo, 61 - lo, s));  // bit 60 orders kNoKey after every box
  DBuf<unsigned> flag;
  OK(flag.alloc(n));
  unique_flags<<<blocks_for(n, 256), 256, 0, s>>>(v.p, n, flag.p);
  OK(cudaGetLastError());
  return select(v, n, flag.p, kept, s);
}

// ---------------------------------------------------------------------------
// refinement, balance and leaves
// ---------------------------------------------------------------------------
__device__ __forceinline__ void anchor_of(uint64_t key, int64_t a[3]) {
  a[0] = compact3(key);
  a[1] = compact3(key >> 1);
  a[2] = compact3(key >> 2);
}

__global__ void split_flags(const uint64_t* keys, long long n, int level, const Predicate p, unsigned* flag) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    int64_t a[3];
    anchor_of(keys[i], a);
    flag[i] = level < p.l_min || (level < p.l_max && geometric_holds(p, a[0], a[1], a[2], level));
  }
}

// wavelet criterion (kind 3): one CTA per box; the field at the box's 13^3 half-node
// points in shared memory, then the largest interpolation failure over the points that
// are not nodes (sums in the fixed order x, then y, then z, each term rounded once)
__global__ void __launch_bounds__(256) wavelet_flags(const uint64_t* keys, long long n, int level, const Predicate p,
                                                     unsigned* flag) {
  __shared__ double F[13 * 13 * 13];
  __shared__ double W[13][7];
  __shared__ double red[256];
  for (long long i = blockIdx.x; i < n; i += gridDim.x) {
    __syncthreads();
    int64_t a[3];
    anchor_of(keys[i], a);
    const int64_t edge = int64_t(1) << (kDepth - level);
    for (int t = threadIdx.x; t < 13 * 7; t += blockDim.x) W[t / 7][t % 7] = wavelet_weight(t / 7, t % 7);
    for (int q = threadIdx.x; q < 13 * 13 * 13; q += blockDim.x)
      F[q] = wavelet_field(p, a, edge, q % 13, (q / 13) % 13, q / 169);
    __syncthreads();
    double worst = 0.0;
    for (int q = threadIdx.x; q < 13 * 13 * 13; q += blockDim.x) {
      const int kx = q % 13, ky = (q / 13) % 13, kz = q / 169;
      if (!((kx | ky | kz) & 1)) continue;
      double vz = 0.0;
      for (int c = 0; c < 7; ++c) {
        double vy = 0.0;
        for (int b = 0; b < 7; ++b) {
          double vx = 0.0;
          for (int aa = 0; aa < 7; ++aa) vx = rn_add(vx, rn_mul(W[kx][aa], F[2 * aa + 26 * b + 338 * c]));
          vy = rn_add(vy, rn_mul(W[ky][b], vx));
        }
        vz = rn_add(vz, rn_mul(W[kz][c], vy));
      }
      const double gap = fabs(rn_sub(F[q], vz));
      if (gap > worst) worst = gap;
    }
    red[threadIdx.x] = worst;
    __syncthreads();
    for (int off = 128; off > 0; off >>= 1) {
      if (threadIdx.x < off && red[threadIdx.x + off] > red[threadIdx.x]) red[threadIdx.x] = red[threadIdx.x + off];
      __syncthreads();
    }
    if (threadIdx.x == 0) flag[i] = level < p.l_min || (level < p.l_max && red[0] > p.eps);
  }
}

__global__ void children_of(const uint64_t* par, long long n, int level, uint64_t* out) {
  const int sh = 3 * (kDepth - level - 1);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < 8 * n; i += (long long)gridDim.x * blockDim.x)
    out[i] = par[i >> 3] + (uint64_t(i & 7) << sh);
}

// the parents (level k - 1) of the 27 same-size boxes around every split box of level k
__global__ void balance_candidates(const uint64_t* split, long long n, int k, uint64_t* out) {
  const int64_t e = int64_t(1) << (kDepth - k);
  const int64_t root = int64_t(1) << kDepth;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < 27 * n; t += (long long)gridDim.x * blockDim.x) {
    const long long i = t / 27;
    const int d = int(t - i * 27);
    int64_t a[3];
    anchor_of(split[i], a);
    const int64_t nb[3] = {a[0] + (d % 3 - 1) * e, a[1] + ((d / 3) % 3 - 1) * e, a[2] + (d / 9 - 1) * e};
    bool inside = true;
    for (int q = 0; q < 3; ++q) inside = inside && nb[q] >= 0 && nb[q] < root;
    const int64_t pe = 2 * e;
    out[t] = inside ? morton3(uint32_t(nb[0] / pe * pe), uint32_t(nb[1] / pe * pe), uint32_t(nb[2] / pe * pe)) : kNoKey;
  }
}

__global__ void leaf_flags(const uint64_t* kids, long long n, const uint64_t* split, long long ns, unsigned* flag) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    flag[i] = !contains(split, ns, kids[i]);
}

// ---------------------------------------------------------------------------
// o2o
// ---------------------------------------------------------------------------
struct LevelSets {
  const uint64_t* leaf[kMaxLevel + 2];
  long long nleaf[kMaxLevel + 2];
  const uint64_t* split[kMaxLevel + 2];
  long long nsplit[kMaxLevel + 2];
  long long off[kMaxLevel + 3];  // level offsets of the leaves (level order)
  int lmax;
};

// level and level-order index of leaf b
__device__ __forceinline__ int level_of(const LevelSets& L, long long b) {
  int l = 0;
  while (l < L.lmax && b >= L.off[l + 1]) ++l;
  return l;
}

// the o2o entry of leaf b in direction d; sets *split_box when the box is split (and its
// 8 children are then looked up by o2o_fill)
__device__ int o2o_entry(const LevelSets& L, long long b, int d, int* bad, bool* split_box, uint64_t* box_key) {
  *split_box = false;
  const int l = level_of(L, b);
  const uint64_t key = L.leaf[l][b - L.off[l]];
  int64_t a[3];
  anchor_of(key, a);
  const int64_t e = int64_t(1) << (kDepth - l), root = int64_t(1) << kDepth;
  const int64_t nb[3] = {a[0] + (d % 3 - 1) * e, a[1] + ((d / 3) % 3 - 1) * e, a[2] + (d / 9 - 1) * e};
  for (int q = 0; q < 3; ++q)
    if (nb[q] < 0 || nb[q] >= root) return -1;
  const uint64_t k = morton3(uint32_t(nb[0]), uint32_t(nb[1]), uint32_t(nb[2]));
  long long at;
  if (contains(L.leaf[l], L.nleaf[l], k, &at)) return int(L.off[l] + at);
  if (l >= 1) {
    const int64_t pe = 2 * e;
    const uint64_t kp = morton3(uint32_t(nb[0] / pe * pe), uint32_t(nb[1] / pe * pe), uint32_t(nb[2] / pe * pe));
    if (contains(L.leaf[l - 1], L.nleaf[l - 1], kp, &at)) return int(L.off[l - 1] + at);
  }
  if (l + 1 <= L.lmax && contains(L.split[l], L.nsplit[l], k)) {
    *split_box = true;
    *box_key = k;
    return -2;
  }
  atomicOr(bad, 1);  // a leaf two or more levels coarser covers the box: never after the balance
  return -1;
}

__global__ void o2o_count(const LevelSets L, long long n, unsigned* cnt, int* bad) {
  for (long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x; b < n; b += (long long)gridDim.x * blockDim.x) {
    unsigned c = 0;
    for (int d = 0; d < 27; ++d) {
      if (d == 13) continue;
      bool sp;
      uint64_t k;
      o2o_entry(L, b, d, bad, &sp, &k);
      c += sp;
    }
    cnt[b] = c;
  }
}

// nbr[b][d]: leaf index (same level or one coarser), -1 outside the domain, or -(2 + f)
// for a split box whose children are fine[f][8] (-1: not a leaf), f in (b, d) order
__global__ void o2o_fill(const LevelSets L, long long n, const unsigned* fpos, int* nbr, int* fine, int* bad) {
  for (long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x; b < n; b += (long long)gridDim.x * blockDim.x) {
    unsigned f = fpos[b];
    const int l = level_of(L, b);
    for (int d = 0; d < 27; ++d) {
      if (d == 13) {
        nbr[b * 27 + d] = int(b);
        continue;
      }
      bool sp;
      uint64_t k;
      int v = o2o_entry(L, b, d, bad, &sp, &k);
      if (sp) {
        const int sh = 3 * (kDepth - l - 1);
        for (int c = 0; c < 8; ++c) {
          long long at;
          const uint64_t ck = k + (uint64_t(c) << sh);
          fine[(long long)f * 8 + c] = contains(L.leaf[l + 1], L.nleaf[l + 1], ck, &at) ? int(L.off[l + 1] + at) : -1;
          const int dd[3] = {d % 3 - 1, (d / 3) % 3 - 1, d / 9 - 1};
          const int cc[3] = {c & 1, (c >> 1) & 1, (c >> 2) & 1};
          bool touches = true;
          for (int q = 0; q < 3; ++q) touches = touches && (dd[q] == 0 || (dd[q] < 0) == (cc[q] == 1));
          if (touches && fine[(long long)f * 8 + c] < 0) atomicOr(bad, 2);  // a finer neighbour two levels finer
        }
        v = -int(2 + f);
        ++f;
      }
      nbr[b * 27 + d] = v;
    }
  }
}

__global__ void decode_leaves(const uint64_t* keys, long long n, int level, int32_t* out /* [n][4] */) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    int64_t a[3];
    anchor_of(keys[i], a);
    out[4 * i + 0] = int32_t(a[0]);
    out[4 * i + 1] = int32_t(a[1]);
    out[4 * i + 2] = int32_t(a[2]);
    out[4 * i + 3] = level;
  }
}

cudaError_t build(const lts_refine_spec& spec, std::vector<Oct>* leaves, Neighbours* nb, int* bad, cudaStream_t s) {
  const Predicate pred = make_predicate(spec);
  const int lmax = spec.l_max;
  std::vector<std::unique_ptr<DBuf<uint64_t>>> split(lmax + 2), lv(lmax + 2);
  std::vector<long long> nsplit(lmax + 2, 0), nleaf(lmax + 2, 0);
  for (int l = 0; l <= lmax + 1; ++l) {
    split[l].reset(new DBuf<uint64_t>());
    lv[l].reset(new DBuf<uint64_t>());
  }
  // refinement, top down
  DBuf<uint64_t> cur;
  OK(cur.alloc(1));
  OK(cudaMemsetAsync(cur.p, 0, sizeof(uint64_t), s));
  long long ncur = 1;
  for (int l = 0; l < lmax && ncur > 0; ++l) {
    DBuf<unsigned> flag;
    OK(flag.alloc(ncur));
    if (pred.kind == 3 && l >= pred.l_min)
      wavelet_flags<<<blocks_for(ncur, 1), 256, 0, s>>>(cur.p, ncur, l, pred, flag.p);
    else
      split_flags<<<blocks_for(ncur, 128), 128, 0, s>>>(cur.p, ncur, l, pred, flag.p);
    OK(cudaGetLastError());
    long long ns = 0;
    OK(select(cur, ncur, flag.p, &ns, s));  // cur now holds the split boxes of level l
    std::swap(split[l]->p, cur.p);
    std::swap(split[l]->n, cur.n);
    nsplit[l] = ns;
    OK(cur.alloc(std::max<long long>(8 * ns, 1)));
    if (ns) {
      children_of<<<blocks_for(8 * ns, 256), 256, 0, s>>>(split[l]->p, ns, l, cur.p);
      OK(cudaGetLastError());
    }
    ncur = 8 * ns;
  }
  // 2:1 balance by closure, finest level first
  for (int k = lmax - 1; k >= 1; --k) {
    if (nsplit[k] == 0) continue;
    const long long nc = 27 * nsplit[k] + nsplit[k - 1];
    DBuf<uint64_t> cand;
    OK(cand.alloc(nc));
    balance_candidates<<<blocks_for(27 * nsplit[k], 256), 256, 0, s>>>(split[k]->p, nsplit[k], k, cand.p);
    OK(cudaGetLastError());
    if (nsplit[k - 1])
      OK(cudaMemcpyAsync(cand.p + 27 * nsplit[k], split[k - 1]->p, sizeof(uint64_t) * nsplit[k - 1],
                         cudaMemcpyDeviceToDevice, s));
    long long kept = 0;
    OK(sort_unique(cand, nc, k - 1, &kept, s));
    std::swap(split[k - 1]->p, cand.p);
    std::swap(split[k - 1]->n, cand.n);
    nsplit[k - 1] = kept;
  }
  // leaves: children of the split boxes of level l - 1 that are not split
  if (nsplit[0] == 0) {
    OK(lv[0]->alloc(1));
    OK(cudaMemsetAsync(lv[0]->p, 0, sizeof(uint64_t), s));
    nleaf[0] = 1;
  }
  for (int l = 1; l <= lmax; ++l) {
    const long long nk = 8 * nsplit[l - 1];
    if (nk == 0) continue;
    OK(lv[l]->alloc(nk));
    children_of<<<blocks_for(nk, 256), 256, 0, s>>>(split[l - 1]->p, nsplit[l - 1], l - 1, lv[l]->p);
    OK(cudaGetLastError());
    DBuf<unsigned> flag;
    OK(flag.alloc(nk));
    leaf_flags<<<blocks_for(nk, 256), 256, 0, s>>>(lv[l]->p, nk, split[l]->p, nsplit[l], flag.p);
    OK(cudaGetLastError());
    OK(select(*lv[l], nk, flag.p, &nleaf[l], s));
  }
  LevelSets L{};
  L.lmax = lmax;
  L.off[0] = 0;
  for (int l = 0; l <= lmax + 1; ++l) {
    L.leaf[l] = lv[l]->p;
    L.nleaf[l] = l <= lmax ? nleaf[l] : 0;
    L.split[l] = split[l]->p;
    L.nsplit[l] = l <= lmax ? nsplit[l] : 0;
    L.off[l + 1] = L.off[l] + L.nleaf[l];
  }
  const long long n = L.off[lmax + 1];
  if (n > (1ll << 31) / 27) return cudaErrorInvalidValue;
  // leaves in level order, to the host
  DBuf<int32_t> dec;
  OK(dec.alloc(4 * n));
  for (int l = 0; l <= lmax; ++l)
    if (nleaf[l]) {
      decode_leaves<<<blocks_for(nleaf[l], 256), 256, 0, s>>>(lv[l]->p, nleaf[l], l, dec.p + 4 * L.off[l]);
      OK(cudaGetLastError());
    }
  leaves->resize(n);
  OK(cudaMemcpyAsync(leaves->data(), dec.p, sizeof(int32_t) * 4 * n, cudaMemcpyDeviceToHost, s));
  // o2o
  DBuf<int> d_bad;
  OK(d_bad.alloc(1));
  OK(cudaMemsetAsync(d_bad.p, 0, sizeof(int), s));
  DBuf<unsigned> cnt, fpos;
  OK(cnt.alloc(n));
  OK(fpos.alloc(n));
  o2o_count<<<blocks_for(n, 128), 128, 0, s>>>(L, n, cnt.p, d_bad.p);
  OK(cudaGetLastError());
  unsigned nfine = 0;
  OK(exclusive_scan(cnt.p, fpos.p, n, &nfine, s));
  DBuf<int> d_nbr, d_fine;
  OK(d_nbr.alloc(27 * n));
  OK(d_fine.alloc(std::max<unsigned>(8u * nfine, 8u)));
  o2o_fill<<<blocks_for(n, 128), 128, 0, s>>>(L, n, fpos.p, d_nbr.p, d_fine.p, d_bad.p);
  OK(cudaGetLastError());
  nb->nbr.resize(27 * n);
  nb->fine.resize(8 * size_t(nfine));
  OK(cudaMemcpyAsync(nb->nbr.data(), d_nbr.p, sizeof(int) * 27 * n, cudaMemcpyDeviceToHost, s));
  if (nfine) OK(cudaMemcpyAsync(nb->fine.data(), d_fine.p, sizeof(int) * 8 * nfine, cudaMemcpyDeviceToHost, s));
  OK(cudaMemcpyAsync(bad, d_bad.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  return cudaStreamSynchronize(s);
}

}  // namespace

// Sec. 3.2.2 - 3.2.4 on the device: leaves in level order and their o2o table.
lts_status device_octree(const lts_refine_spec& spec, std::vector<Oct>* leaves, Neighbours* nb, std::string* err) {
  static_assert(sizeof(Oct) == 4 * sizeof(int32_t), "Oct is (x, y, z, level)");
  cudaStream_t s = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  int bad = 0;
  if (e == cudaSuccess) e = build(spec, leaves, nb, &bad, s);
  if (s) cudaStreamDestroy(s);
  if (e != cudaSuccess) {
    *err = std::string("octree_build: ") + cudaGetErrorString(e);
    return LTS_ECUDA;
  }
  if (bad) {
    *err = "octree_build: the balanced tree failed its neighbour check (code " + std::to_string(bad) + ")";
    return LTS_EINTERNAL;
  }
  return LTS_OK;
}

}  // namespace ltsoct
