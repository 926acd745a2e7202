// Host emulation of the lfbp tile code -- TEST INFRASTRUCTURE.
//
// Compiles the device tile functions of lfbp_device.cuh as ordinary C++ with
// checked stand-ins for the GPU primitives, and runs every tile of a plan
// sequentially (the lanes of 1, 2, 3 or 8 producer warps, then consumer threads) so that the
// CPU tests can check, before any GPU run, that
//   * every bulk copy is 16-byte aligned, a multiple of 16 bytes, reads only
//     inside the input array and writes only inside its stage,
//   * the bytes announced with expect_tx equal the bytes copied,
//   * every shared-memory read is inside the stage and every global store is
//     inside the output array and aligned,
//   * every output byte is written exactly once,
// and compare the result with the CPU oracle.
#include <cstddef>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <vector>

#define __device__
#define __host__
#define __forceinline__ inline
#define __noinline__
#define LFBP_HOST_EMULATION 1

struct uint4 {
  unsigned x, y, z, w;
};
struct uint2 {
  unsigned x, y;
};
static inline uint2 make_uint2(unsigned x, unsigned y) { return uint2{x, y}; }
static inline uint4 make_uint4(unsigned x, unsigned y, unsigned z, unsigned w) {
  return uint4{x, y, z, w};
}

namespace {
const unsigned char* g_in = nullptr;
size_t g_in_bytes = 0;
unsigned char* g_out = nullptr;
size_t g_out_bytes = 0;
unsigned char* g_counts = nullptr;
unsigned char* g_stage = nullptr;
size_t g_stage_bytes = 0;
// the tile's row-base table: a second shared-memory region, mapped to
// emulated addresses kTabBase + byte offset
constexpr uint32_t kTabBase = 0x40000000u;
unsigned char* g_tab = nullptr;
size_t g_tab_bytes = 0;
unsigned long long g_expect = 0, g_copied = 0, g_arrive = 0;
long g_errors = 0;
char g_msg[512] = {0};

void err(const char* what, long long a, long long b) {
  if (g_errors++ == 0) std::snprintf(g_msg, sizeof(g_msg), "%s (%lld, %lld)", what, a, b);
}
}  // namespace

static inline uint32_t __umulhi(uint32_t a, uint32_t b) {
  return (uint32_t)(((uint64_t)a * (uint64_t)b) >> 32);
}
static inline void __syncwarp() {}
static inline unsigned __ldg(const unsigned* p) {
  const unsigned char* c = (const unsigned char*)p;
  if (c < g_in || c + 4 > g_in + g_in_bytes || ((uintptr_t)c & 3)) err("ldg32 out of range", c - g_in, 0);
  return *p;
}
static inline unsigned short __ldg(const unsigned short* p) {
  const unsigned char* c = (const unsigned char*)p;
  if (c < g_in || c + 2 > g_in + g_in_bytes || ((uintptr_t)c & 1)) err("ldg16 out of range", c - g_in, 0);
  return *p;
}
namespace lfbp {
static inline uint32_t smem_addr(const void* p) {
  const unsigned char* c = (const unsigned char*)p;
  if (c >= g_tab && c < g_tab + g_tab_bytes) return kTabBase + (uint32_t)(c - g_tab);
  if (c < g_stage || c > g_stage + g_stage_bytes) err("smem_addr outside stage", c - g_stage, 0);
  return (uint32_t)(c - g_stage);
}
static inline void fence_proxy_async_smem() {}
static inline void mbar_expect_tx(uint32_t, uint32_t bytes) { g_expect += bytes; }
static inline void mbar_arrive(uint32_t) { ++g_arrive; }
static inline void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t) {
  const unsigned char* s = (const unsigned char*)src;
  if (bytes == 0 || (bytes & 15)) err("bulk size not a positive multiple of 16", bytes, 0);
  if (((uintptr_t)s & 15) || (dst & 15)) err("bulk copy misaligned", (uintptr_t)s & 15, dst & 15);
  if (s < g_in || s + bytes > g_in + g_in_bytes) err("bulk copy reads outside input", s - g_in, bytes);
  if ((size_t)dst + bytes > g_stage_bytes) err("bulk copy writes outside stage", dst, bytes);
  if (g_errors == 0) std::memcpy(g_stage + dst, s, bytes);
  g_copied += bytes;
}
// 16-byte cp.async (load/store path): same checks as a bulk copy of 16 bytes
static inline void cp_async16(uint32_t dst, const void* src) {
  const unsigned char* s = (const unsigned char*)src;
  if (((uintptr_t)s & 15) || (dst & 15)) err("cp.async misaligned", (uintptr_t)s & 15, dst & 15);
  if (s < g_in || s + 16 > g_in + g_in_bytes) err("cp.async reads outside input", s - g_in, 16);
  if ((size_t)dst + 16 > g_stage_bytes) err("cp.async writes outside stage", dst, 16);
  if (g_errors == 0) std::memcpy(g_stage + dst, s, 16);
  g_copied += 16;
}
static inline void emu_smem_check(long long byte_off) {
  if (byte_off < 0 || (size_t)byte_off >= g_stage_bytes) err("smem read outside stage", byte_off, 0);
}
static inline void count_store(const unsigned char* p, size_t n) {
  if (p < g_out || p + n > g_out + g_out_bytes) {
    err("store outside output", p - g_out, (long long)n);
    return;
  }
  for (size_t i = 0; i < n; ++i) g_counts[(p - g_out) + i]++;
}
template <class T>
static inline T lds(uint32_t addr) {
  T v;
  if (addr >= kTabBase) {
    const size_t off = addr - kTabBase;
    if (off + sizeof(T) > g_tab_bytes || (off & 3)) {
      err("lds outside the row-base table", (long long)off, (long long)g_tab_bytes);
      return (T)0;
    }
    std::memcpy(&v, g_tab + off, sizeof(T));
    return v;
  }
  if ((size_t)addr + sizeof(T) > g_stage_bytes || (addr & (sizeof(T) - 1))) {
    err("lds outside stage or misaligned", addr, (long long)g_stage_bytes);
    return (T)0;
  }
  std::memcpy(&v, g_stage + addr, sizeof(T));
  return v;
}
template <class T, int OFF>
static inline T lds_off(uint32_t addr) {
  return lds<T>(addr + OFF);
}
static inline uint2 lds64(uint32_t addr) {
  uint2 v{0, 0};
  if (addr >= kTabBase || (size_t)addr + 8 > g_stage_bytes || (addr & 7)) {
    err("8-byte lds outside stage or misaligned", addr, (long long)g_stage_bytes);
    return v;
  }
  std::memcpy(&v, g_stage + addr, 8);
  return v;
}
static inline uint4 lds128(uint32_t addr) {
  uint4 v{0, 0, 0, 0};
  if (addr >= kTabBase || (size_t)addr + 16 > g_stage_bytes || (addr & 15)) {
    err("16-byte lds outside stage or misaligned", addr, (long long)g_stage_bytes);
    return v;
  }
  std::memcpy(&v, g_stage + addr, 16);
  return v;
}
template <class T>
static inline void st_global(T* p, T v) {
  if ((uintptr_t)p & (sizeof(T) - 1)) err("store misaligned", (long long)((uintptr_t)p & 15), (long long)sizeof(T));
  count_store((unsigned char*)p, sizeof(T));
  if (g_errors == 0) *p = v;
}
}  // namespace lfbp
#define LFBP_SMEM_CHECK(idx) emu_smem_check((long long)(idx) * ES)

#include "lfbp_device.cuh"

using namespace lfbp;

extern "C" const char* emu_message() { return g_msg; }

// The stripe consumer of one tile with the lanes of each warp run in lock
// step: per warp step and stripe, the four lanes of the group load and cut
// out their windows, exchange them through arrays with the same per-lane
// stage functions the kernel uses between its shuffles, and store; then the
// edge pass, lane by lane.
template <int ES, int S, bool MASK>
static void emu_stripes(const TileCtx& c, int nwarps, int rot) {
  for (int w = 0; w < nwarps; ++w) {
    int first = (w - rot) % nwarps;
    if (first < 0) first += nwarps;
    for (int u = first; u < c.nsteps_s; u += nwarps)
      for (int gs = 0; gs < 8; ++gs) {
        int item = u * 8 + gs;
        const bool ok = item < c.nitems_s;
        if (!ok) item = c.nitems_s - 1;
        StripeStream st[4];
        StripePos sp[4];
        for (int g = 0; g < 4; ++g) {
          sp[g] = stripe_pos<S>(c, item);
          stripe_begin<ES>(c, sp[g], g, st[g]);
        }
        static_for<0, S>([&](auto ic) {
          constexpr int i = decltype(ic)::value;
          uint32_t x[4][ES == 4 ? 4 : 2];
          for (int g = 0; g < 4; ++g) stripe_window<ES, i>(c, st[g], x[g]);
          if constexpr (ES == 4) {
            uint32_t snd[4][2], rcv[2];
            for (int g = 0; g < 4; ++g) xs_a32(x[g], g, snd[g]);
            for (int g = 0; g < 4; ++g) {
              rcv[0] = snd[g ^ 2][0];
              rcv[1] = snd[g ^ 2][1];
              xr_a32(x[g], g, rcv);
            }
            for (int g = 0; g < 4; ++g) xs_b32(x[g], g, snd[g]);
            for (int g = 0; g < 4; ++g) {
              rcv[0] = snd[g ^ 1][0];
              rcv[1] = snd[g ^ 1][1];
              xr_b32(x[g], g, rcv);
            }
          } else {
            uint32_t snd[4];
            for (int g = 0; g < 4; ++g) snd[g] = xs_a16(x[g], g);
            for (int g = 0; g < 4; ++g) xr_a16(x[g], g, snd[g ^ 2]);
            for (int g = 0; g < 4; ++g) snd[g] = xs_b16(x[g], g);
            for (int g = 0; g < 4; ++g) xr_b16(x[g], g, snd[g ^ 1]);
          }
          for (int g = 0; g < 4; ++g) stripe_store<ES, i, MASK>(c, sp[g], g, ok, x[g]);
        });
      }
  }
  for (int w = 0; w < nwarps; ++w)
    for (int lane = 0; lane < 32; ++lane) stripe_edges<ES, MASK>(c, w, nwarps, lane, rot);
}

template <int ES, bool MASK>
static void emu_stripes_s(const TileCtx& c, int nwarps, int rot) {
  switch (c.S) {
    case 1: emu_stripes<ES, 1, MASK>(c, nwarps, rot); break;
    case 2: emu_stripes<ES, 2, MASK>(c, nwarps, rot); break;
    case 3: emu_stripes<ES, 3, MASK>(c, nwarps, rot); break;
    case 4: emu_stripes<ES, 4, MASK>(c, nwarps, rot); break;
    case 5: emu_stripes<ES, 5, MASK>(c, nwarps, rot); break;
    default: err("stripe length beyond the instances", c.S, 0); break;
  }
}

static void emu_stripes_ctx(const TileCtx& c, int nwarps, int rot) {
  if (c.es == 4) {
    if (c.mode == 0) emu_stripes_s<4, false>(c, nwarps, rot);
    else emu_stripes_s<4, true>(c, nwarps, rot);
  } else {
    if (c.mode == 0) emu_stripes_s<2, false>(c, nwarps, rot);
    else emu_stripes_s<2, true>(c, nwarps, rot);
  }
}

// Runs every tile of every depth of one array through the tile code.
// Returns the number of violations (0 = clean); stats[0] = tiles, stats[1] =
// bytes copied by bulk copies, stats[2] = max tile bytes, stats[3] = tiles
// whose context selects the chunk path, stats[4] = tiles that took the stripe
// path, stats[5] = tiles that took the pair path (pair, then stripe, then the
// chunk or element-walk path).  nthr = consumer warps.
extern "C" long emu_run(const unsigned char* in, unsigned char* out, unsigned char* counts,
                        int Nx, int Ny, int Nz, const int* Ks, const int* Kt, int es, int mode,
                        int target, int nthr, unsigned long long* stats) {
  g_errors = 0;
  g_msg[0] = 0;
  size_t total = 0;
  std::vector<size_t> off(Nz + 1, 0);
  for (int z = 0; z < Nz; ++z) {
    off[z + 1] = off[z] + (size_t)Nx * Ny * Ks[z] * Kt[z];
  }
  total = off[Nz] * es;
  g_in = in;
  g_in_bytes = total;
  g_out = out;
  g_out_bytes = total;
  g_counts = counts;
  const unsigned char* safe_end = in + (total & ~(size_t)15);
  unsigned long long tiles = 0, copied = 0, maxb = 0, nfast = 0, nstripe = 0, npair = 0;
  for (int z = 0; z < Nz && g_errors == 0; ++z) {
    DepthTiling d = tile_depth(Ny, Ks[z], Kt[z], es, target);
    if ((unsigned long long)d.max_tile_bytes > maxb) maxb = d.max_tile_bytes;
    TileDesc base;
    std::memset(&base, 0, sizeof(base));
    base.off_bytes = off[z] * es;
    base.Nx = (unsigned short)Nx;
    base.Ny = (unsigned short)Ny;
    base.Ks = (unsigned short)Ks[z];
    base.Kt = (unsigned short)Kt[z];
    base.P = (unsigned short)d.P;
    base.flags = (unsigned char)((es == 2 ? 1 : 0) | (mode << 1) | ((Ks[z] % 2 == 0) << 3) |
                                 ((Kt[z] % 2 == 0) << 4));
    if ((d.P - (long long)Ks[z] * Kt[z]) % (16 / es) != 0) err("pitch not congruent to Ks*Kt", d.P, 0);
    if (d.P < d.V + 2 * (16 / es) - 2) err("pitch too small", d.P, d.V);
    std::vector<unsigned char> stage((size_t)d.max_tile_bytes + 64);
    for (int ub = 0; ub < d.nU; ++ub)
      for (int p = 0; p < Nx; ++p)
        for (int vb = 0; vb < d.nV; ++vb) {
          TileDesc td = base;
          td.p = (unsigned short)p;
          td.u0 = (unsigned short)(ub * d.J);
          td.v0 = (unsigned short)(vb * d.V);
          td.nrows = (unsigned short)lfbp_min(d.J, Ks[z] - ub * d.J);
          td.ncols = (unsigned short)lfbp_min(d.V, Kt[z] - vb * d.V);
          const unsigned tile_bytes = td.nrows * row_pitch(Ny, d.P, es) * es;
          if ((int)tile_bytes > d.max_tile_bytes) err("tile larger than its depth's maximum", tile_bytes, d.max_tile_bytes);
          std::memset(stage.data(), 0xA5, stage.size());
          g_stage = stage.data();
          g_stage_bytes = tile_bytes;
          g_expect = g_copied = g_arrive = 0;
          const unsigned char* in_depth = in + base.off_bytes;
          unsigned char* out_depth = out + base.off_bytes;
          // the copies of a tile are shared by np producer warps; cycle np
          // through the counts the kernels use
          static const int kNp[4] = {1, 2, 3, 8};
          const int np = kNp[tiles % 4];
          for (int pw = 0; pw < np; ++pw)
            for (int lane = 0; lane < 32; ++lane)
              g_expect += tile_copies(td, in_depth, safe_end, stage.data(), 0, lane, pw, np, true);
          for (int pw = 0; pw < np; ++pw)
            for (int lane = 0; lane < 32; ++lane)
              tile_copies(td, in_depth, safe_end, stage.data(), 0, lane, pw, np, false);
          if (g_expect != g_copied) err("expect_tx bytes differ from bytes copied", g_expect, g_copied);
          // the load/store-path copies (tile_copies_lsu) must fill a second
          // stage with exactly the same bytes, poison included
          {
            std::vector<unsigned char> stage2(stage.size());
            std::memset(stage2.data(), 0xA5, stage2.size());
            const unsigned long long copied_tma = g_copied;
            g_copied = 0;
            g_stage = stage2.data();
            for (int pw = 0; pw < np; ++pw)
              for (int lane = 0; lane < 32; ++lane)
                tile_copies_lsu(td, in_depth, safe_end, stage2.data(), lane, pw, np);
            if (g_copied != copied_tma) err("cp.async bytes differ from bulk-copy bytes", g_copied, copied_tma);
            if (std::memcmp(stage.data(), stage2.data(), stage.size()) != 0)
              err("cp.async stage differs from the bulk-copy stage", (long long)tiles, 0);
            g_stage = stage.data();
            g_copied = copied_tma;
          }
          const int nwarps = nthr;  // here: number of consumer warps
          TileCtx ctx;
          // table entries past nrows stay poisoned: reading them is an error
          std::vector<int> tab(kMaxTileRows + 1, 0x7f7f7f7f);
          g_tab = (unsigned char*)tab.data();
          g_tab_bytes = (size_t)(td.nrows + 1) * sizeof(int);
          const int cls = (ub + 1 == d.nU ? 1 : 0) + (vb + 1 == d.nV ? 2 : 0);
          td.shape = (unsigned short)cls;
          const TileShape shp = depth_shape(d, Nx, Ny, Ks[z], Kt[z], es, base.flags, cls);
          // the shape class must describe this tile
          if (shp.nrows != td.nrows || shp.ncols != td.ncols) err("shape class does not fit the tile", shp.nrows, td.nrows);
          make_ctx(ctx, td, &shp, stage.data(), in_depth, out_depth, tab.data());
          nfast += ctx.fast ? 1 : 0;
          nstripe += ctx.stripe ? 1 : 0;
          npair += ctx.pair ? 1 : 0;
          const int nsteps = ctx.pair ? (ctx.punits + 31) / 32
                                      : (ctx.stripe ? ctx.nsteps_s : (ctx.fast ? ctx.nunits : ctx.items));
          const int rot = (int)((tiles * (unsigned long long)nsteps) % nwarps);
          if (ctx.stripe) {
            emu_stripes_ctx(ctx, nwarps, rot);
          } else {
            for (int w = 0; w < nwarps; ++w)
              for (int lane = 0; lane < 32; ++lane) gather_tile_ctx(ctx, w, nwarps, lane, rot);
          }
          g_tab = nullptr;  // the table dies with this tile
          g_tab_bytes = 0;
          ++tiles;
          copied += g_copied;
          if (g_errors) break;
        }
  }
  if (stats) {
    stats[0] = tiles;
    stats[1] = copied;
    stats[2] = maxb;
    stats[3] = nfast;
    stats[4] = nstripe;
    stats[5] = npair;
  }
  return g_errors;
}
