// Voxel hash shared by the ICP map, the scan downsampling and the anchor
// maintenance: packed integer voxel keys, an open-addressing table with linear
// probing, and the map buffer (header, table, points grouped by voxel) that
// vpgs_icp_build_map writes.  The voxel of a coordinate x for an edge v is
// floor(x / v) in float32 with the correctly rounded division.
#pragma once

#include <cmath>

#include "common.cuh"
#include "prims.cuh"

namespace vpgs {
namespace {

constexpr unsigned long long kEmptyKey = ~0ull;
constexpr uint32_t kNoSlot = 0xffffffffu;
constexpr int kVoxRange = 1 << 20;  // |voxel index| < 2^20 on every axis
constexpr uint32_t kMapMagic = 0x49435056u;

struct MapHeader {
    uint32_t magic, cap, n_voxels, status;
    int64_t n;
    float voxel;
    uint32_t ticket, total, pad[7];
};
static_assert(sizeof(MapHeader) == 64, "map header is 64 bytes");

// map: a = first point, b = point count; downsampling: a = lowest index
struct __align__(16) VoxEntry {
    unsigned long long key;
    uint32_t a, b;
};


inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

inline uint32_t table_cap(int64_t n) {
    uint64_t c = 1024;
    while (c < 2 * (uint64_t)n) c <<= 1;
    return (uint32_t)c;
}

struct MapLayout {
    uint32_t cap;
    size_t off_tab, off_pts, off_slot, off_look, n_look, total;
};

inline MapLayout map_layout(int64_t n) {
    MapLayout L;
    L.cap = table_cap(n);
    size_t o = sizeof(MapHeader);
    L.off_tab = o;
    o += sizeof(VoxEntry) * (size_t)L.cap;
    L.off_pts = o;
    o += sizeof(float4) * (size_t)n;
    L.off_slot = o;
    o = align_up(o + sizeof(uint32_t) * (size_t)n, 16);
    L.off_look = o;
    L.n_look = (size_t)std::max<int64_t>(scan_blocks(L.cap), 1);
    o += sizeof(unsigned long long) * L.n_look;
    L.total = o;
    return L;
}


// ---------------------------------------------------------------------------
// voxels and the hash
// ---------------------------------------------------------------------------
VPGS_D bool voxel_index(float x, float v, int &i) {
    const float q = floorf(__fdiv_rn(x, v));
    if (!(q >= -(float)kVoxRange && q < (float)kVoxRange)) return false;  // also rejects NaN
    i = (int)q;
    return true;
}

VPGS_D bool in_voxel_range(int i) { return i >= -kVoxRange && i < kVoxRange; }

VPGS_D unsigned long long pack_voxel(int ix, int iy, int iz) {
    return ((unsigned long long)(uint32_t)(ix + kVoxRange) << 42) |
           ((unsigned long long)(uint32_t)(iy + kVoxRange) << 21) | (unsigned long long)(uint32_t)(iz + kVoxRange);
}

// the splitmix64 finaliser (Steele, Lea and Flood, "Fast splittable
// pseudorandom number generators", 2014) as the hash of a packed voxel
VPGS_D uint32_t hash_slot(unsigned long long k, uint32_t mask) {
    k ^= k >> 30;
    k *= 0xbf58476d1ce4e5b9ull;
    k ^= k >> 27;
    k *= 0x94d049bb133111ebull;
    k ^= k >> 31;
    return (uint32_t)k & mask;
}

// Slot of `key`, claimed if absent; kNoSlot if the table is full (it never
// is: the capacity is at least twice the number of keys).
VPGS_D uint32_t insert_voxel(VoxEntry *tab, uint32_t mask, unsigned long long key, bool &fresh) {
    uint32_t h = hash_slot(key, mask);
    for (uint32_t p = 0; p <= mask; ++p) {
        const unsigned long long cur = __ldcg(&tab[h].key);
        if (cur == key) {
            fresh = false;
            return h;
        }
        if (cur == kEmptyKey) {
            const unsigned long long prev = atomicCAS(&tab[h].key, kEmptyKey, key);
            if (prev == kEmptyKey || prev == key) {
                fresh = prev == kEmptyKey;
                return h;
            }
        }
        h = (h + 1) & mask;
    }
    fresh = false;
    return kNoSlot;
}

// The entry of `key` (one 16-byte load per probe); count 0 when absent.
VPGS_D VoxEntry find_entry(const VoxEntry *tab, uint32_t mask, unsigned long long key) {
    uint32_t h = hash_slot(key, mask);
    for (uint32_t p = 0; p <= mask; ++p) {
        const ulonglong2 e = *reinterpret_cast<const ulonglong2 *>(&tab[h]);
        if (e.x == key) return VoxEntry{e.x, (uint32_t)e.y, (uint32_t)(e.y >> 32)};
        if (e.x == kEmptyKey) break;
        h = (h + 1) & mask;
    }
    return VoxEntry{kEmptyKey, 0u, 0u};
}


struct MapView {
    const MapHeader *hdr;
    const VoxEntry *tab;
    const float4 *pts;
    uint32_t mask;
    int64_t n;
    float voxel;
};


// distance from x to the slab [lo, lo + v) of voxel i (0 inside)
VPGS_D float slab_gap(int i, float v, float x) {
    const float lo = (float)i * v;
    return fmaxf(fmaxf(lo - x, x - (lo + v)), 0.f);
}


inline bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }
inline bool pos_finite(float x) { return std::isfinite(x) && x > 0.f; }


inline bool map_args_ok(const void *map, size_t map_bytes, int64_t n_map, float voxel) {
    if (!map || !aligned16(map) || n_map < 0 || n_map > (int64_t(1) << 30) || !pos_finite(voxel)) return false;
    return map_bytes >= map_layout(n_map).total;
}

inline MapView map_view(const void *map, int64_t n_map, float voxel) {
    const MapLayout L = map_layout(n_map);
    const char *b = static_cast<const char *>(map);
    MapView m;
    m.hdr = reinterpret_cast<const MapHeader *>(b);
    m.tab = reinterpret_cast<const VoxEntry *>(b + L.off_tab);
    m.pts = reinterpret_cast<const float4 *>(b + L.off_pts);
    m.mask = L.cap - 1;
    m.n = n_map;
    m.voxel = voxel;
    return m;
}


}  // namespace
}  // namespace vpgs

namespace vpgs {
namespace {

// True when some point of the map lies closer than r to c: (dx^2 + dy^2) +
// dz^2 < r^2 in float32, d = m - c, over the 27 voxels around c (exact for
// r <= the map's voxel edge).  Called by all 32 lanes of a warp with the same
// c: lane k < 27 probes neighbour k, then the lanes stride each live voxel's
// points and stop at the first hit.
VPGS_D bool warp_map_any_within(const MapView &map, float cx, float cy, float cz, float r) {
    const int lane = threadIdx.x & 31;
    const float v = map.voxel;
    int ix = 0, iy = 0, iz = 0;
    const bool ok = voxel_index(cx, v, ix) && voxel_index(cy, v, iy) && voxel_index(cz, v, iz);
    const float r2 = __fmul_rn(r, r);
    const float lim = r + 1e-4f + 1e-6f * fmaxf(fmaxf(fabsf(cx), fabsf(cy)), fabsf(cz));
    uint32_t start = 0, cnt = 0;
    if (ok && lane < 27) {
        const int nx = ix + lane % 3 - 1, ny = iy + (lane / 3) % 3 - 1, nz = iz + lane / 9 - 1;
        if (in_voxel_range(nx) && in_voxel_range(ny) && in_voxel_range(nz)) {
            const float gx = slab_gap(nx, v, cx), gy = slab_gap(ny, v, cy), gz = slab_gap(nz, v, cz);
            if (gx * gx + gy * gy + gz * gz <= lim * lim) {
                const VoxEntry e = find_entry(map.tab, map.mask, pack_voxel(nx, ny, nz));
                start = e.a;
                cnt = e.b;
            }
        }
    }
    uint32_t live = __ballot_sync(0xffffffffu, cnt > 0);
    while (live) {
        const int k = __ffs(live) - 1;
        live &= live - 1;
        const uint32_t s0 = __shfl_sync(0xffffffffu, start, k), c = __shfl_sync(0xffffffffu, cnt, k);
        for (uint32_t q0 = 0; q0 < c; q0 += 32) {
            bool hit = false;
            if (q0 + lane < c) {
                const float4 m = map.pts[s0 + q0 + lane];
                const float ex = __fsub_rn(m.x, cx), ey = __fsub_rn(m.y, cy), ez = __fsub_rn(m.z, cz);
                const float d2 = __fadd_rn(__fadd_rn(__fmul_rn(ex, ex), __fmul_rn(ey, ey)), __fmul_rn(ez, ez));
                hit = d2 < r2;
            }
            if (__any_sync(0xffffffffu, hit)) return true;
        }
    }
    return false;
}

// float32 centre (k + 1/2) v of voxel k
VPGS_D float voxel_centre(int k, float v) { return __fmul_rn(__fadd_rn((float)k, 0.5f), v); }

// A map header that matches the host's view of the buffer (device check).
VPGS_D bool map_header_ok(const MapView &map) {
    const MapHeader *h = map.hdr;
    return h->magic == kMapMagic && h->n == map.n && h->cap == map.mask + 1 &&
           __float_as_uint(h->voxel) == __float_as_uint(map.voxel);
}

}  // namespace
}  // namespace vpgs
