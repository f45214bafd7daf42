// fe_tiles.cu -- element tiles of the fused element + patch kernels (host side).
//
// The exact gradient g_i = sum_{(T,l) in patch(i)} r_{T,l} - b_i (Sec. 6.2, eqs. dJdvn and
// dWFv) needs, for every node, the local forces of all elements of its patch.  The fused
// kernels evaluate one tile -- a contiguous range of device-order elements (the elements lie
// along the Morton curve of their centroids, so a range is a compact piece of the mesh) --
// per thread block, keep the tile's local forces in shared memory and sum there the patch of
// every node whose whole patch lies in the tile.  Only the nodes on the tile's surface, whose
// patches span several tiles, leave a partial sum per tile in global memory; a second small
// kernel adds those partials in tile order.  Every sum has a fixed order, so results are
// bitwise reproducible, and no atomics touch the gradient.
//
// This file builds, once per mesh, on the host:
//   - the tile cut: consecutive elements, in groups of kTileAlign, until kTileElems elements
//     or tile_max_nodes(dim) distinct nodes;
//   - per tile, its nodes (sorted by id) and, per element, the tile-local ids of its vertices;
//   - per tile, a local patch CSR: the entries (e, l) of each tile node in element order, as
//     local slots; the element kernel writes r_{T,l} to local slot (e, l);
//   - the owner of each node's b_i v_i term (the first tile holding the node);
//   - the partial slots of the shared nodes: numbered tile by tile (a tile writes its
//     partials to consecutive slots) and listed per node in tile order.
// Nodes in no element form node-only tiles at the end (their gradient is -b_i, 0 on
// Dirichlet dofs).
#include <algorithm>
#include <vector>

#include "fe_internal.cuh"

namespace fe {

void free_tiles(fe_ctx* c) {
  dev_free(c, &c->tile_ebeg, (size_t)c->n_tiles + 1);
  dev_free(c, &c->tile_nbeg, (size_t)c->n_tiles + 1);
  dev_free(c, &c->tile_node, (size_t)c->n_tnodes);
  dev_free(c, &c->tile_elem, (size_t)c->ne);
  dev_free(c, &c->tile_snode, (size_t)c->n_shared);
  dev_free(c, &c->tile_sbeg, (size_t)c->n_shared + 1);
  dev_free(c, &c->tile_spart, (size_t)c->n_tpart);
  dev_free(c, &c->tile_part, (size_t)c->n_tpart * (c->d > 0 ? c->d : 1));
  dev_free(c, &c->tile_epart, 2 * (size_t)c->n_tiles);
  dev_free(c, &c->tile_bvp, (size_t)(c->nn + kThreads - 1) / kThreads);
  c->n_tiles = c->n_tnodes = c->n_shared = c->n_tpart = 0;
}

fe_status build_tiles(fe_ctx* c) {
  free_tiles(c);
  const int dim = c->dim, K = dim + 1;
  const int64_t nn = c->nn, ne = c->ne;
  const int nmax = tile_max_nodes(dim);
  std::vector<int32_t> E((size_t)ne * K);
  if (ne > 0) {
    fe_status st = cuda_check(cudaMemcpy(E.data(), c->elems, sizeof(int32_t) * E.size(), cudaMemcpyDeviceToHost),
                              "tile build: read elements");
    if (st) return st;
  }
  auto node_of = [&](int64_t e, int l) { return E[(size_t)l * ne + e]; };

  // pass 1: the cut, and the nodes of every tile
  std::vector<int32_t> ebeg{0}, nbeg{0}, tnode;
  std::vector<int32_t> stamp(nn, -1), ntile(nn, 0);
  std::vector<int32_t> cur;
  int32_t t = 0;
  int in_tile = 0;
  auto close_tile = [&](int64_t e_end) {
    std::sort(cur.begin(), cur.end());
    for (int32_t n : cur) {
      tnode.push_back(n);
      ntile[n]++;
    }
    nbeg.push_back((int32_t)tnode.size());
    ebeg.push_back((int32_t)e_end);
    cur.clear();
    ++t;
    in_tile = 0;
  };
  // elements join a tile in groups of kTileAlign (so that every tile starts on a multiple
  // of kTileAlign); a group's new nodes are counted once (a node repeated in the group is
  // counted on its first appearance)
  std::vector<int32_t> fresh_nodes;
  for (int64_t e = 0; e < ne;) {
    const int64_t ge = std::min<int64_t>(e + kTileAlign, ne);
    fresh_nodes.clear();
    for (int64_t q = e; q < ge; ++q)
      for (int l = 0; l < K; ++l) {
        const int32_t n = node_of(q, l);
        if (stamp[n] != t && std::find(fresh_nodes.begin(), fresh_nodes.end(), n) == fresh_nodes.end())
          fresh_nodes.push_back(n);
      }
    if (in_tile + (ge - e) > kTileElems || (int)(cur.size() + fresh_nodes.size()) > nmax) {
      close_tile(e);
      continue;
    }
    for (int32_t n : fresh_nodes) {
      stamp[n] = t;
      cur.push_back(n);
    }
    in_tile += (int)(ge - e);
    e = ge;
  }
  if (in_tile > 0) close_tile(ne);
  // node-only tiles for nodes in no element
  for (int64_t i = 0; i < nn; ++i)
    if (ntile[i] == 0) {
      cur.push_back((int32_t)i);
      if ((int)cur.size() == nmax) close_tile(ne);
    }
  if (!cur.empty()) close_tile(ne);
  if (t == 0) close_tile(ne);  // an empty mesh still has one (empty) tile for the energy
  const int64_t ntiles = t, ntn = (int64_t)tnode.size();

  // shared nodes (in more than one tile): their partials, listed per node in tile order
  std::vector<int32_t> sidx(nn, -1), snode, sbeg{0};
  for (int64_t i = 0; i < nn; ++i)
    if (ntile[i] > 1) {
      sidx[i] = (int32_t)snode.size();
      snode.push_back((int32_t)i);
      sbeg.push_back(sbeg.back() + ntile[i]);
    }
  const int64_t nshared = (int64_t)snode.size(), npart = sbeg.back();
  // partial slots are numbered tile by tile (the tile's shared nodes in node order), so that
  // a tile writes its partials to consecutive slots; spart lists each node's slots
  std::vector<int32_t> spart((size_t)npart);
  int32_t next_part = 0;

  // pass 2: local ids, local slots, node records
  std::vector<uint4> telem((size_t)ne);
  std::vector<int4> trec((size_t)ntn);
  std::vector<int32_t> loc(nn, -1), srank(nshared, 0);
  std::vector<uint8_t> owned(nn, 0);
  std::vector<int32_t> cnt, pos;
  for (int64_t tt = 0; tt < ntiles; ++tt) {
    const int32_t k0 = nbeg[tt], nt = nbeg[tt + 1] - k0;
    const int32_t e0 = ebeg[tt], e1 = ebeg[tt + 1];
    cnt.assign(nt, 0);
    for (int32_t k = 0; k < nt; ++k) loc[tnode[k0 + k]] = k;
    for (int32_t e = e0; e < e1; ++e)
      for (int l = 0; l < K; ++l) cnt[loc[node_of(e, l)]]++;
    pos.assign(nt, 0);
    int32_t run = 0;
    for (int32_t k = 0; k < nt; ++k) {
      pos[k] = run;
      const int32_t i = tnode[k0 + k];
      int32_t dst = -1;
      if (ntile[i] > 1) {
        dst = next_part++;
        spart[sbeg[sidx[i]] + srank[sidx[i]]++] = dst;
      }
      const int32_t owner = owned[i] ? 0 : 1;
      owned[i] = 1;
      const int32_t src = c->perm_h.empty() ? i : c->perm_h[i];
      trec[k0 + k] = make_int4(i, src, run | (cnt[k] << 16), ((dst + 1) << 1) | owner);
      run += cnt[k];
    }
    for (int32_t e = e0; e < e1; ++e) {
      uint32_t lid[4] = {0, 0, 0, 0}, sl[4] = {0, 0, 0, 0};
      for (int l = 0; l < K; ++l) {
        const int32_t k = loc[node_of(e, l)];
        lid[l] = (uint32_t)k;
        sl[l] = (uint32_t)pos[k]++;
      }
      telem[e] = make_uint4(lid[0] | (lid[1] << 16), lid[2] | (lid[3] << 16), sl[0] | (sl[1] << 16),
                            sl[2] | (sl[3] << 16));
    }
  }

  fe_status st;
  if ((st = dev_alloc(c, &c->tile_ebeg, (size_t)ntiles + 1)) || (st = dev_alloc(c, &c->tile_nbeg, (size_t)ntiles + 1)) ||
      (st = dev_alloc(c, &c->tile_node, (size_t)ntn)) || (st = dev_alloc(c, &c->tile_elem, (size_t)ne)) ||
      (st = dev_alloc(c, &c->tile_snode, (size_t)nshared)) || (st = dev_alloc(c, &c->tile_sbeg, (size_t)nshared + 1)) ||
      (st = dev_alloc(c, &c->tile_spart, (size_t)npart)) ||
      (st = dev_alloc(c, &c->tile_part, (size_t)npart * (c->d > 0 ? c->d : 1))) ||
      (st = dev_alloc(c, &c->tile_epart, 2 * (size_t)ntiles)) ||
      (st = dev_alloc(c, &c->tile_bvp, (size_t)(nn + kThreads - 1) / kThreads))) {
    c->n_tiles = ntiles;
    c->n_tnodes = ntn;
    c->n_shared = nshared;
    c->n_tpart = npart;
    free_tiles(c);
    return st;
  }
  c->n_tiles = ntiles;
  c->n_tnodes = ntn;
  c->n_shared = nshared;
  c->n_tpart = npart;
  cudaMemcpy(c->tile_ebeg, ebeg.data(), sizeof(int32_t) * ebeg.size(), cudaMemcpyHostToDevice);
  cudaMemcpy(c->tile_nbeg, nbeg.data(), sizeof(int32_t) * nbeg.size(), cudaMemcpyHostToDevice);
  if (ntn > 0) cudaMemcpy(c->tile_node, trec.data(), sizeof(int4) * trec.size(), cudaMemcpyHostToDevice);
  if (ne > 0) cudaMemcpy(c->tile_elem, telem.data(), sizeof(uint4) * telem.size(), cudaMemcpyHostToDevice);
  if (nshared > 0) cudaMemcpy(c->tile_snode, snode.data(), sizeof(int32_t) * snode.size(), cudaMemcpyHostToDevice);
  cudaMemcpy(c->tile_sbeg, sbeg.data(), sizeof(int32_t) * sbeg.size(), cudaMemcpyHostToDevice);
  if (npart > 0) cudaMemcpy(c->tile_spart, spart.data(), sizeof(int32_t) * spart.size(), cudaMemcpyHostToDevice);
  return cuda_check(cudaGetLastError(), "tile build: upload");
}

}  // namespace fe
