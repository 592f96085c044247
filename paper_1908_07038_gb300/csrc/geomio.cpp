// Geometry cache: the host grid, mesh and dual of an fvm written to a file
// and read back, so that a large grid's host build (seconds at O1280) is
// done once.  See geometry.h.
//
// File layout (little-endian): the 8 bytes "ATLGEOM1", a uint32 format
// version (1) and a uint32 zero; the scalar block (int64 values in a fixed
// order, then the radius and the 8 projection parameters as doubles); then
// every array as {uint64 count, uint32 element size, uint32 zero, data} in a
// fixed order; last, a 64-bit FNV-1a hash (over 8-byte words) of every byte
// before it.
#include <cstdio>
#include <cstring>
#include <vector>

#include "geometry.h"

namespace atlasgb {

namespace {

constexpr char kMagic[8] = {'A', 'T', 'L', 'G', 'E', 'O', 'M', '1'};
constexpr uint32_t kVersion = 1;
constexpr uint64_t kFnvOffset = 1469598103934665603ull;

// FNV-1a over the 64-bit little-endian words of each written piece, then
// its remaining bytes (the pieces are the same when reading back)
uint64_t mix(uint64_t h, const void* p, size_t n) {
  const unsigned char* c = static_cast<const unsigned char*>(p);
  size_t k = 0;
  for (; k + 8 <= n; k += 8) {
    uint64_t w;
    std::memcpy(&w, c + k, 8);
    h = (h ^ w) * 1099511628211ull;
  }
  for (; k < n; ++k) h = (h ^ c[k]) * 1099511628211ull;
  return h;
}

struct Writer {
  FILE* f;
  uint64_t h = kFnvOffset;
  bool ok = true;
  void raw(const void* p, size_t n) {
    if (!ok || n == 0) return;
    h = mix(h, p, n);
    ok = std::fwrite(p, 1, n, f) == n;
  }
  template <typename T> void scalar(T v) { raw(&v, sizeof(T)); }
  template <typename T> void vec(const std::vector<T>& v) {
    scalar<uint64_t>(v.size());
    scalar<uint32_t>(sizeof(T));
    scalar<uint32_t>(0);
    raw(v.data(), v.size() * sizeof(T));
  }
};

struct Reader {
  FILE* f;
  uint64_t h = kFnvOffset;
  uint64_t left;  // bytes of the file not read yet
  bool ok = true;
  void raw(void* p, size_t n) {
    if (!ok || n == 0) return;
    if (n > left) {
      ok = false;
      return;
    }
    ok = std::fread(p, 1, n, f) == n;
    left -= n;
    if (ok) h = mix(h, p, n);
  }
  template <typename T> T scalar() {
    T v{};
    raw(&v, sizeof(T));
    return v;
  }
  template <typename T> void vec(std::vector<T>& v) {
    const uint64_t n = scalar<uint64_t>();
    const uint32_t es = scalar<uint32_t>();
    (void)scalar<uint32_t>();
    if (!ok || es != sizeof(T) || n > left / sizeof(T)) {
      ok = false;
      return;
    }
    v.resize(static_cast<size_t>(n));
    raw(v.data(), static_cast<size_t>(n) * sizeof(T));
  }
};

template <typename T> bool sized(const std::vector<T>& v, int64_t n) { return static_cast<int64_t>(v.size()) == n; }

}  // namespace

bool save_geometry(const Grid& g, const Mesh& m, const Dual& d, const char* path, const char** why) {
  FILE* f = std::fopen(path, "wb");
  if (!f) {
    if (why) *why = "cannot open the file for writing";
    return false;
  }
  Writer w{f};
  w.raw(kMagic, sizeof(kMagic));
  w.scalar<uint32_t>(kVersion);
  w.scalar<uint32_t>(0);
  for (int64_t v : {static_cast<int64_t>(g.N), static_cast<int64_t>(g.nlat), static_cast<int64_t>(g.octahedral),
                    g.nnodes, static_cast<int64_t>(g.projection), static_cast<int64_t>(g.nx), m.nedges, m.ntri})
    w.scalar<int64_t>(v);
  w.scalar<double>(d.R);
  for (double p : g.proj_params) w.scalar<double>(p);
  w.vec(g.pl);
  w.vec(g.off);
  w.vec(g.colat);
  w.vec(g.lat);
  w.vec(g.lonlat);
  w.vec(g.xy);
  w.vec(g.h);
  w.vec(m.e2n);
  w.vec(m.is_pole);
  w.vec(m.n2e_ptr);
  w.vec(m.n2e);
  w.vec(m.n2e_sign);
  w.vec(m.tri);
  w.vec(m.side_off);
  w.vec(m.side_lat);
  w.vec(m.mid_lat);
  w.vec(d.S);
  w.vec(d.V);
  w.vec(d.coslat);
  w.vec(d.pole_nphi);
  w.vec(d.A);
  w.vec(d.Sb);
  const uint64_t hash = w.h;
  w.raw(&hash, sizeof(hash));
  const bool closed = std::fclose(f) == 0;
  if (!w.ok || !closed) {
    if (why) *why = "write failed";
    return false;
  }
  return true;
}

bool load_geometry(const char* path, Grid& g, Mesh& m, Dual& d, const char** why) {
  auto bad = [&](const char* w) {
    if (why) *why = w;
    return false;
  };
  FILE* f = std::fopen(path, "rb");
  if (!f) return bad("cannot open the file");
  std::fseek(f, 0, SEEK_END);
  const long size = std::ftell(f);
  std::fseek(f, 0, SEEK_SET);
  if (size < static_cast<long>(sizeof(kMagic) + 8 + sizeof(uint64_t))) {
    std::fclose(f);
    return bad("not a geometry file (too short)");
  }
  // the trailing hash is read apart
  Reader r{f, kFnvOffset, static_cast<uint64_t>(size) - sizeof(uint64_t)};
  char magic[8];
  r.raw(magic, sizeof(magic));
  const uint32_t version = r.scalar<uint32_t>();
  (void)r.scalar<uint32_t>();
  if (!r.ok || std::memcmp(magic, kMagic, sizeof(kMagic)) != 0) {
    std::fclose(f);
    return bad("not a geometry file");
  }
  if (version != kVersion) {
    std::fclose(f);
    return bad("unsupported geometry file version");
  }
  int64_t sc[8];
  for (int64_t& v : sc) v = r.scalar<int64_t>();
  g.N = static_cast<int>(sc[0]);
  g.nlat = static_cast<int>(sc[1]);
  g.octahedral = sc[2] != 0;
  g.nnodes = sc[3];
  g.projection = static_cast<int>(sc[4]);
  g.nx = static_cast<int>(sc[5]);
  m.nedges = sc[6];
  m.ntri = sc[7];
  d.R = r.scalar<double>();
  for (double& p : g.proj_params) p = r.scalar<double>();
  r.vec(g.pl);
  r.vec(g.off);
  r.vec(g.colat);
  r.vec(g.lat);
  r.vec(g.lonlat);
  r.vec(g.xy);
  r.vec(g.h);
  r.vec(m.e2n);
  r.vec(m.is_pole);
  r.vec(m.n2e_ptr);
  r.vec(m.n2e);
  r.vec(m.n2e_sign);
  r.vec(m.tri);
  r.vec(m.side_off);
  r.vec(m.side_lat);
  r.vec(m.mid_lat);
  r.vec(d.S);
  r.vec(d.V);
  r.vec(d.coslat);
  r.vec(d.pole_nphi);
  r.vec(d.A);
  r.vec(d.Sb);
  const uint64_t computed = r.h;
  uint64_t stored = 0;
  const bool tail_ok = r.ok && r.left == 0 && std::fread(&stored, 1, sizeof(stored), f) == sizeof(stored);
  std::fclose(f);
  if (!tail_ok) return bad("truncated or malformed geometry file");
  if (stored != computed) return bad("geometry file checksum mismatch (corrupted)");
  const int64_t V = g.nnodes, E = m.nedges, T = m.ntri;
  const bool regional = g.projection >= 0;
  if (V <= 0 || E <= 0 || T <= 0 || g.nlat <= 0 || !(d.R > 0) || !sized(g.pl, g.nlat) || !sized(g.off, g.nlat + 1) ||
      !sized(g.lonlat, 2 * V) || !sized(m.e2n, 2 * E) || !sized(m.is_pole, E) || !sized(m.n2e_ptr, V + 1) ||
      !sized(m.n2e, 2 * E) || !sized(m.n2e_sign, 2 * E) || !sized(m.tri, 3 * T) || !sized(d.S, 2 * E) ||
      !sized(d.V, V) || !sized(d.coslat, V) || !sized(d.pole_nphi, V) ||
      (regional && (!sized(g.xy, 2 * V) || !sized(g.h, 2 * V) || !sized(d.A, V) || !sized(d.Sb, 2 * E))))
    return bad("inconsistent array sizes in the geometry file");
  if (g.off[0] != 0 || g.off[g.nlat] != V) return bad("inconsistent row offsets in the geometry file");
  m.grid = &g;
  return true;
}

}  // namespace atlasgb
