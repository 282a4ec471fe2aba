// Lattice geometry: even-odd neighbour tables and the sub-lattice regions of the
// multisplitting block operator.
//
// Paper Sec. 2.2 (parity = (x+y+z+t) mod 2) and Sec. 2.3: the Dirichlet block
// operator A_s = P_s D_PC^+ D_PC P_s keeps the "snake" paths that leave the block
// and come back. D_PC has two hops, so D_PC P_s x lives on the even sites within
// lattice distance 2 of the block, and the odd intermediates of both halves live
// within distance 1. Those sites, found with periodic (wrapped) distances, are
// the block's region; every block of one shape has the same region in
// block-relative coordinates because block origins are even.
#include <algorithm>
#include <array>
#include <unordered_map>

#include "dwf_internal.cuh"

namespace dwf {

static inline int lex(const int c[4], const int L[4]) {
  return ((c[3] * L[2] + c[2]) * L[1] + c[1]) * L[0] + c[0];
}

void build_geometry(Geometry &g, const int dims[4]) {
  for (int m = 0; m < 4; ++m) g.dims[m] = dims[m];
  g.V4 = dims[0] * dims[1] * dims[2] * dims[3];
  g.Vh = g.V4 / 2;
  for (int p = 0; p < 2; ++p) {
    g.nbr[p].assign((size_t)g.Vh * 8, -1);
    for (int h = 0; h < g.Vh; ++h) {
      int idx0 = 2 * h;
      int c[4];
      c[0] = idx0 % dims[0];
      c[1] = (idx0 / dims[0]) % dims[1];
      c[2] = (idx0 / (dims[0] * dims[1])) % dims[2];
      c[3] = idx0 / (dims[0] * dims[1] * dims[2]);
      c[0] += (p + c[1] + c[2] + c[3]) & 1;  // the site of parity p in the pair
      for (int mu = 0; mu < 4; ++mu) {
        for (int dir = 0; dir < 2; ++dir) {
          int n[4] = {c[0], c[1], c[2], c[3]};
          n[mu] = (n[mu] + (dir == 0 ? 1 : dims[mu] - 1)) % dims[mu];
          g.nbr[p][(size_t)h * 8 + 2 * mu + dir] = lex(n, dims) >> 1;
        }
      }
    }
  }
}

// Periodic distance of local coordinate u (relative to the block origin) from
// the block interval [0, bl) in a direction of extent L.
static inline int dist1(int u, int bl, int L) {
  if (u < bl) return 0;
  return std::min(u - bl + 1, L - u);
}

// Which side of the block interval u lies on: 0 inside, 1 above (u >= bl),
// 2 below (wrapped round, nearer the block's start).
static inline int side1(int u, int bl, int L) {
  if (u < bl) return 0;
  return (u - bl + 1 <= L - u) ? 1 : 2;
}

void build_block_geometry(BlockGeometry &bg, const int dims[4], const int block[4]) {
  int nb[4];
  for (int m = 0; m < 4; ++m) {
    DWF_REQUIRE(block[m] > 0 && block[m] % 2 == 0 && dims[m] % block[m] == 0,
                DWF_ERR_INVALID_ARG, "block extents must be even and divide the lattice");
    bg.block[m] = block[m];
    nb[m] = dims[m] / block[m];
  }
  bg.nblocks = nb[0] * nb[1] * nb[2] * nb[3];

  // candidate local coordinates per direction (distance <= 2)
  std::vector<int> cand[4];
  for (int m = 0; m < 4; ++m) {
    std::vector<char> seen(dims[m], 0);
    for (int u = 0; u < dims[m]; ++u)
      if (dist1(u, block[m], dims[m]) <= 2 && !seen[u]) {
        seen[u] = 1;
        cand[m].push_back(u);
      }
  }
  struct Site {
    int u[4];
    int d, par, lexl;
    int face;  // side1 of the four coordinates, two bits each
  };
  std::vector<Site> sites;
  for (int t : cand[3])
    for (int z : cand[2])
      for (int y : cand[1])
        for (int x : cand[0]) {
          Site s;
          s.u[0] = x; s.u[1] = y; s.u[2] = z; s.u[3] = t;
          s.d = dist1(x, block[0], dims[0]) + dist1(y, block[1], dims[1]) +
                dist1(z, block[2], dims[2]) + dist1(t, block[3], dims[3]);
          if (s.d > 2) continue;
          s.par = (x + y + z + t) & 1;
          s.lexl = lex(s.u, dims);
          s.face = 0;
          for (int m = 0; m < 4; ++m) s.face |= side1(s.u[m], block[m], dims[m]) << (2 * m);
          sites.push_back(s);
        }
  std::vector<Site> ev, od;
  for (auto &s : sites) {
    if (s.par == 0) ev.push_back(s);
    else if (s.d <= 1) od.push_back(s);
  }
  // by distance (the block's own sites first, then the rings), and within a
  // ring by face, so that the sites of one warp share their pattern of
  // neighbours inside the region (a ring site has only one or two)
  auto key = [](const Site &a, const Site &b) {
    if (a.d != b.d) return a.d < b.d;
    if (a.face != b.face) return a.face < b.face;
    return a.lexl < b.lexl;
  };
  std::sort(ev.begin(), ev.end(), key);
  std::sort(od.begin(), od.end(), key);
  bg.n_e2 = (int)ev.size();
  bg.n_o1 = (int)od.size();
  bg.n_b = (int)std::count_if(ev.begin(), ev.end(), [](const Site &s) { return s.d == 0; });
  bg.n_e1 = (int)std::count_if(ev.begin(), ev.end(), [](const Site &s) { return s.d <= 1; });
  bg.n_ob = (int)std::count_if(od.begin(), od.end(), [](const Site &s) { return s.d == 0; });
  bg.n_comb = bg.n_e2 + bg.n_o1;

  std::unordered_map<int, int> ev_idx, od_idx;
  for (int i = 0; i < bg.n_e2; ++i) ev_idx[ev[i].lexl] = i;
  for (int i = 0; i < bg.n_o1; ++i) od_idx[od[i].lexl] = i;

  auto nb_lex = [&](const Site &s, int mu, int dir) {
    int n[4] = {s.u[0], s.u[1], s.u[2], s.u[3]};
    n[mu] = (n[mu] + (dir == 0 ? 1 : dims[mu] - 1)) % dims[mu];
    return lex(n, dims);
  };
  bg.nbr_oe.assign((size_t)bg.n_o1 * 8, -1);
  for (int i = 0; i < bg.n_o1; ++i)
    for (int mu = 0; mu < 4; ++mu)
      for (int dir = 0; dir < 2; ++dir) {
        auto it = ev_idx.find(nb_lex(od[i], mu, dir));
        if (it != ev_idx.end()) bg.nbr_oe[(size_t)i * 8 + 2 * mu + dir] = it->second;
      }
  bg.nbr_eo.assign((size_t)bg.n_e2 * 8, -1);
  for (int i = 0; i < bg.n_e2; ++i)
    for (int mu = 0; mu < 4; ++mu)
      for (int dir = 0; dir < 2; ++dir) {
        auto it = od_idx.find(nb_lex(ev[i], mu, dir));
        if (it != od_idx.end()) bg.nbr_eo[(size_t)i * 8 + 2 * mu + dir] = it->second;
      }

  bg.gsite.assign((size_t)bg.nblocks * bg.n_comb, 0);
  bg.gmap_b.assign((size_t)bg.nblocks * bg.n_b, 0);
  for (int b = 0; b < bg.nblocks; ++b) {
    int bc[4] = {b % nb[0], (b / nb[0]) % nb[1], (b / (nb[0] * nb[1])) % nb[2],
                 b / (nb[0] * nb[1] * nb[2])};
    auto glob = [&](const Site &s) {
      int c[4];
      for (int m = 0; m < 4; ++m) c[m] = (bc[m] * block[m] + s.u[m]) % dims[m];
      return lex(c, dims);
    };
    for (int i = 0; i < bg.n_e2; ++i) bg.gsite[(size_t)b * bg.n_comb + i] = glob(ev[i]);
    for (int i = 0; i < bg.n_o1; ++i) bg.gsite[(size_t)b * bg.n_comb + bg.n_e2 + i] = glob(od[i]);
    for (int i = 0; i < bg.n_b; ++i) bg.gmap_b[(size_t)b * bg.n_b + i] = glob(ev[i]) >> 1;
  }
}

}  // namespace dwf
