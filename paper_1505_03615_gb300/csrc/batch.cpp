// batch.cpp -- concatenation of separately built hierarchies into one batch.
//
// Many meshes of uneven size are solved together: every kernel of a V-cycle
// then covers the rows of all meshes at once, and one persistent launch drives
// the whole batch.  Levels are aligned at the finest: batch level D - k holds
// level inst_D - k of every mesh that has one.  On a batch level the rows that
// are smoothed (meshes with a coarser level below) come first, ordered by
// colour, then mesh, then the mesh's own order, so one colour is still one
// contiguous range without couplings inside it; rows of meshes whose coarsest
// level this is follow, mesh by mesh, for the dense coarse solve.
#include <algorithm>
#include <numeric>

#include "hier.h"

namespace lbmg {

namespace {

// A batch of one mesh has the layout below with identity row and entry maps, so the mesh's
// own arrays are taken over instead of being remapped entry by entry.
int adopt_single(HostHierarchy &P, HostHierarchy &B, std::string &err) {
    if ((int64_t)P.nfrag * 36 > (int64_t)UINT32_MAX) { err = "batch too large"; return 1; }
    B = HostHierarchy();
    B.ninst = 1;
    B.split = P.split;
    B.D = P.D;
    B.d0 = P.d0;
    const int nu = P.lev[P.D].ndof;
    B.inst_D = {P.D};
    B.inst_d0 = {P.d0};
    B.inst_voff = {0};
    B.inst_toff = {0};
    B.inst_uoff = {0};
    B.inst_nfine = {nu};
    B.inst_sigma = {P.sigma};
    B.inst_S = {P.S};
    B.inst_center = {P.center[0], P.center[1], P.center[2]};
    B.nv = P.nv;
    B.nt = P.nt;
    B.nfrag = P.nfrag;
    B.S = P.S;
    B.sigma = P.sigma;
    for (int a = 0; a < 3; a++) B.center[a] = P.center[a];
    B.Vg = std::move(P.Vg);
    B.F = std::move(P.F);
    B.tri_normal = std::move(P.tri_normal);
    B.frag_tri = std::move(P.frag_tri);
    B.frag_vox = std::move(P.frag_vox);
    B.frag_pstart = std::move(P.frag_pstart);
    B.frag_poly = std::move(P.frag_poly);
    B.frag_dof = std::move(P.frag_dof);
    B.arp = std::move(P.arp);
    B.aidx = std::move(P.aidx);
    B.rrp = std::move(P.rrp);
    B.ridx = std::move(P.ridx);
    B.vdof = std::move(P.vdof);
    B.vw = std::move(P.vw);
    B.frag_scale.assign(P.nfrag, P.sigma * P.sigma);
    B.fperm.resize(nu);
    std::iota(B.fperm.begin(), B.fperm.end(), 0);
    B.lev = std::move(P.lev);
    for (int d = 0; d <= B.D; d++) {
        HostLevel &L = B.lev[d];
        // the (corner, triangle) lookup tables serve the build only
        std::vector<CornerTri>().swap(L.ct);
        std::vector<int32_t>().swap(L.ct_dof);
        if (d < B.d0) continue;
        L.inst.assign(L.ndof, 0);
        for (int c = 0; c <= 8; c++) L.colour_all[c] = L.colour_start[c];
        if (d == B.d0) {
            // the coarsest level is one dense block and is not smoothed
            for (int c = 0; c <= 8; c++) L.colour_start[c] = 0;
            L.ns = 0;
            L.coarse = {0, 0, L.ndof};
        } else {
            L.ns = L.ndof;
        }
    }
    B.seg.assign(16, 0);
    const HostLevel &LF = B.lev[B.D];
    if (B.D > B.d0) {
        for (int c = 0; c < 8; c++) { B.seg[2 * c] = LF.colour_start[c]; B.seg[2 * c + 1] = LF.colour_start[c + 1]; }
    } else {
        B.seg[1] = LF.ndof;
    }
    return 0;
}

}  // namespace

int combine_batch(std::vector<HostHierarchy> &parts, HostHierarchy &B, std::string &err) {
    const int ni = (int)parts.size();
    if (ni < 1) { err = "empty batch"; return 1; }
    if (ni == 1) return adopt_single(parts[0], B, err);
    B = HostHierarchy();
    B.ninst = ni;
    B.split = parts[0].split;
    int Lmax = 0;
    for (auto &p : parts) Lmax = std::max(Lmax, p.D - p.d0 + 1);
    // a single mesh keeps its own depths; a batch counts levels from the finest
    B.D = ni == 1 ? parts[0].D : Lmax - 1;
    B.d0 = B.D - (Lmax - 1);
    if (B.d0 < 0 || B.D > kMaxDepth) { err = "batch depth out of range"; return 1; }
    auto real = [&](int i, int dB) { return parts[i].D - (B.D - dB); };

    // instance tables and concatenated geometry
    B.inst_D.resize(ni); B.inst_d0.resize(ni); B.inst_voff.resize(ni); B.inst_toff.resize(ni);
    B.inst_uoff.resize(ni); B.inst_nfine.resize(ni); B.inst_sigma.resize(ni); B.inst_S.resize(ni);
    B.inst_center.resize(3 * (size_t)ni);
    std::vector<int64_t> foff(ni), poff(ni);
    int64_t nv = 0, nt = 0, nf = 0, np = 0, nu = 0;
    for (int i = 0; i < ni; i++) {
        HostHierarchy &P = parts[i];
        B.inst_D[i] = P.D; B.inst_d0[i] = P.d0;
        B.inst_voff[i] = (int32_t)nv; B.inst_toff[i] = (int32_t)nt; B.inst_uoff[i] = (int32_t)nu;
        B.inst_nfine[i] = P.lev[P.D].ndof;
        B.inst_sigma[i] = P.sigma; B.inst_S[i] = P.S;
        for (int a = 0; a < 3; a++) B.inst_center[3 * i + a] = P.center[a];
        foff[i] = nf; poff[i] = np;
        nv += P.nv; nt += P.nt; nf += P.nfrag; np += P.frag_pstart[P.nfrag]; nu += P.lev[P.D].ndof;
    }
    if (nf * 36 > (int64_t)UINT32_MAX || nv > INT32_MAX || nt > INT32_MAX) { err = "batch too large"; return 1; }
    B.nv = (int)nv; B.nt = (int)nt; B.nfrag = (int)nf;
    B.S = parts[0].S; B.sigma = parts[0].sigma;
    for (int a = 0; a < 3; a++) B.center[a] = parts[0].center[a];
    B.Vg.resize(3 * nv); B.F.resize(3 * nt); B.tri_normal.resize(3 * nt);
    B.frag_tri.resize(nf); B.frag_vox.resize(3 * nf); B.frag_pstart.resize(nf + 1);
    B.frag_poly.resize(3 * np); B.frag_scale.resize(nf);
    B.frag_pstart[0] = 0;
    for (int i = 0; i < ni; i++) {
        HostHierarchy &P = parts[i];
        const int64_t vo = B.inst_voff[i], to = B.inst_toff[i], fo = foff[i];
        std::copy(P.Vg.begin(), P.Vg.end(), B.Vg.begin() + 3 * vo);
        std::copy(P.tri_normal.begin(), P.tri_normal.end(), B.tri_normal.begin() + 3 * to);
        std::copy(P.frag_poly.begin(), P.frag_poly.end(), B.frag_poly.begin() + 3 * poff[i]);
#pragma omp parallel for schedule(static)
        for (int64_t q = 0; q < 3 * (int64_t)P.nt; q++) B.F[3 * to + q] = P.F[q] + (int32_t)vo;
#pragma omp parallel for schedule(static)
        for (int f = 0; f < P.nfrag; f++) {
            B.frag_tri[fo + f] = P.frag_tri[f] + (int32_t)to;
            for (int a = 0; a < 3; a++) B.frag_vox[3 * (fo + f) + a] = P.frag_vox[3 * (size_t)f + a];
            B.frag_pstart[fo + f + 1] = (int32_t)(poff[i] + P.frag_pstart[f + 1]);
            B.frag_scale[fo + f] = P.sigma * P.sigma;
        }
    }

    B.lev.assign(B.D + 1, HostLevel());
    // row and stored-entry maps of the level just processed (the finer one for the next)
    std::vector<std::vector<int32_t>> rmapF(ni), nmapF(ni), rmap(ni), nmap(ni);
    for (int dB = B.D; dB >= B.d0; dB--) {
        HostLevel &L = B.lev[dB];
        L.d = dB;
        for (int i = 0; i < ni; i++) { rmap[i].clear(); nmap[i].clear(); }
        int row = 0;
        auto smooth = [&](int i) { int r = real(i, dB); return r > parts[i].d0 && r <= parts[i].D; };
        auto coarse = [&](int i) { return real(i, dB) == parts[i].d0; };
        for (int i = 0; i < ni; i++)
            if (smooth(i) || coarse(i)) rmap[i].assign(parts[i].lev[real(i, dB)].ndof, -1);
        if (dB == B.D) B.seg.assign(16 * (size_t)ni, 0);
        for (int c = 0; c < 8; c++) {
            L.colour_start[c] = row;
            for (int i = 0; i < ni; i++) {
                if (!smooth(i)) continue;
                const HostLevel &P = parts[i].lev[real(i, dB)];
                if (dB == B.D) B.seg[2 * (8 * (size_t)i + c)] = row;
                for (int a = P.colour_start[c]; a < P.colour_start[c + 1]; a++) rmap[i][a] = row++;
                if (dB == B.D) B.seg[2 * (8 * (size_t)i + c) + 1] = row;
            }
        }
        L.colour_start[8] = row;
        L.ns = row;
        for (int i = 0; i < ni; i++) {
            if (!coarse(i)) continue;
            const HostLevel &P = parts[i].lev[real(i, dB)];
            L.coarse.push_back(i);
            L.coarse.push_back(row);
            L.coarse.push_back(P.ndof);
            if (dB == B.D) { B.seg[2 * (8 * (size_t)i)] = row; B.seg[2 * (8 * (size_t)i) + 1] = row + P.ndof; }
            for (int a = 0; a < P.ndof; a++) rmap[i][a] = row++;
        }
        L.ndof = row;
        L.corner.assign(3 * (size_t)row, 0);
        L.mintri.assign(row, 0);
        L.inst.assign(row, 0);
        std::vector<int32_t> src_i(row), src_a(row);
        for (int i = 0; i < ni; i++)
            for (int a = 0; a < (int)rmap[i].size(); a++) {
                const int r = rmap[i][a];
                if (r < 0) { err = "internal: unmapped row"; return 1; }
                const HostLevel &P = parts[i].lev[real(i, dB)];
                src_i[r] = i; src_a[r] = a;
                for (int k = 0; k < 3; k++) L.corner[3 * (size_t)r + k] = P.corner[3 * (size_t)a + k];
                L.mintri[r] = P.mintri[a];
                L.inst[r] = i;
            }
        // CSR with remapped, re-sorted columns; nmap: local stored entry -> batch stored entry
        L.rp.assign(row + 1, 0);
        for (int r = 0; r < row; r++) {
            const HostLevel &P = parts[src_i[r]].lev[real(src_i[r], dB)];
            L.rp[r + 1] = L.rp[r] + (P.rp[src_a[r] + 1] - P.rp[src_a[r]]);
        }
        L.ci.assign(L.rp[row], 0);
        for (int i = 0; i < ni; i++)
            if (!rmap[i].empty()) nmap[i].assign(parts[i].lev[real(i, dB)].ci.size(), -1);
#pragma omp parallel
        {
            std::vector<std::pair<int32_t, int32_t>> tmp;
#pragma omp for schedule(dynamic, 256)
            for (int r = 0; r < row; r++) {
                const int i = src_i[r], a = src_a[r];
                const HostLevel &P = parts[i].lev[real(i, dB)];
                tmp.clear();
                for (int k = P.rp[a]; k < P.rp[a + 1]; k++) tmp.push_back({rmap[i][P.ci[k]], k});
                std::sort(tmp.begin(), tmp.end());
                for (size_t q = 0; q < tmp.size(); q++) {
                    L.ci[L.rp[r] + q] = tmp[q].first;
                    nmap[i][tmp[q].second] = L.rp[r] + (int32_t)q;
                }
            }
        }
        if (dB == B.D) {
            // finest: fragments, assembly and right-hand-side lists, vertex evaluation, user order
            B.frag_dof.resize(8 * (size_t)nf);
            for (int i = 0; i < ni; i++) {
                const HostHierarchy &P = parts[i];
#pragma omp parallel for schedule(static)
                for (size_t q = 0; q < P.frag_dof.size(); q++)
                    B.frag_dof[8 * (size_t)foff[i] + q] = rmap[i][P.frag_dof[q]];
            }
            const int64_t nnz = L.rp[row];
            B.arp.assign(nnz + 1, 0);
            for (int i = 0; i < ni; i++) {
                const HostHierarchy &P = parts[i];
#pragma omp parallel for schedule(static)
                for (size_t k = 0; k < nmap[i].size(); k++) B.arp[nmap[i][k] + 1] = P.arp[k + 1] - P.arp[k];
            }
            for (int64_t s = 0; s < nnz; s++) B.arp[s + 1] += B.arp[s];
            B.aidx.assign(B.arp[nnz], 0);
            for (int i = 0; i < ni; i++) {
                const HostHierarchy &P = parts[i];
                const uint32_t fo36 = (uint32_t)(36 * foff[i]);
#pragma omp parallel for schedule(static)
                for (size_t k = 0; k < nmap[i].size(); k++) {
                    int64_t o = B.arp[nmap[i][k]];
                    for (int64_t q = P.arp[k]; q < P.arp[k + 1]; q++) B.aidx[o++] = P.aidx[q] + fo36;
                }
            }
            B.rrp.assign(row + 1, 0);
            for (int r = 0; r < row; r++) {
                const HostHierarchy &P = parts[src_i[r]];
                B.rrp[r + 1] = B.rrp[r] + (P.rrp[src_a[r] + 1] - P.rrp[src_a[r]]);
            }
            B.ridx.assign(B.rrp[row], 0);
#pragma omp parallel for schedule(static)
            for (int r = 0; r < row; r++) {
                const HostHierarchy &P = parts[src_i[r]];
                int64_t o = B.rrp[r];
                for (int64_t q = P.rrp[src_a[r]]; q < P.rrp[src_a[r] + 1]; q++)
                    B.ridx[o++] = P.ridx[q] + (uint32_t)(8 * foff[src_i[r]]);
            }
            B.vdof.assign(8 * nv, -1);
            B.vw.assign(8 * nv, 0.0);
            for (int i = 0; i < ni; i++) {
                const HostHierarchy &P = parts[i];
#pragma omp parallel for schedule(static)
                for (size_t q = 0; q < P.vdof.size(); q++) {
                    const size_t o = 8 * (size_t)B.inst_voff[i] + q;
                    B.vdof[o] = P.vdof[q] >= 0 ? rmap[i][P.vdof[q]] : -1;
                    B.vw[o] = P.vw[q];
                }
            }
            B.fperm.assign(nu, 0);
            for (int i = 0; i < ni; i++)
                for (int a = 0; a < (int)rmap[i].size(); a++) B.fperm[B.inst_uoff[i] + a] = rmap[i][a];
        } else {
            // this level as the coarse side of dB+1: children, Galerkin lists; parents of dB+1
            HostLevel &Lf = B.lev[dB + 1];
            L.crp.assign(row + 1, 0);
            for (int r = 0; r < row; r++) {
                const HostLevel &P = parts[src_i[r]].lev[real(src_i[r], dB)];
                L.crp[r + 1] = L.crp[r] + (P.crp[src_a[r] + 1] - P.crp[src_a[r]]);
            }
            L.cch.assign(L.crp[row], 0);
#pragma omp parallel for schedule(static)
            for (int r = 0; r < row; r++) {
                const int i = src_i[r];
                const HostLevel &P = parts[i].lev[real(i, dB)];
                int o = L.crp[r];
                for (int q = P.crp[src_a[r]]; q < P.crp[src_a[r] + 1]; q++) {
                    const uint32_t e = P.cch[q];
                    L.cch[o++] = (uint32_t)rmapF[i][e & kPackMask] | (e & ~kPackMask);
                }
            }
            const int64_t nnz = L.rp[row];
            L.grp.assign(nnz + 1, 0);
            for (int i = 0; i < ni; i++) {
                if (rmap[i].empty()) continue;
                const HostLevel &P = parts[i].lev[real(i, dB)];
#pragma omp parallel for schedule(static)
                for (size_t k = 0; k < nmap[i].size(); k++) L.grp[nmap[i][k] + 1] = P.grp[k + 1] - P.grp[k];
            }
            for (int64_t s = 0; s < nnz; s++) L.grp[s + 1] += L.grp[s];
            L.gidx.assign(L.grp[nnz], 0);
            int too_large = 0;
            for (int i = 0; i < ni; i++) {
                if (rmap[i].empty()) continue;
                const HostLevel &P = parts[i].lev[real(i, dB)];
#pragma omp parallel for schedule(static) reduction(| : too_large)
                for (size_t k = 0; k < nmap[i].size(); k++) {
                    int64_t o = L.grp[nmap[i][k]];
                    for (int64_t q = P.grp[k]; q < P.grp[k + 1]; q++) {
                        const uint32_t e = P.gidx[q];
                        const int32_t idx = nmapF[i][e & kGalMask];
                        too_large |= (uint32_t)idx > kGalMask;
                        L.gidx[o++] = (uint32_t)idx | (e & ~kGalMask);
                    }
                }
            }
            if (too_large) { err = "batch level too large for packed Galerkin lists"; return 1; }
            Lf.par.assign(8 * (size_t)Lf.ndof, -1);
            Lf.npar_log2.assign(Lf.ndof, 0);
            for (int i = 0; i < ni; i++) {
                if (rmapF[i].empty() || rmap[i].empty()) continue;
                const HostLevel &P = parts[i].lev[real(i, dB + 1)];
                if (P.par.empty()) continue;
#pragma omp parallel for schedule(static)
                for (int a = 0; a < P.ndof; a++) {
                    const int r = rmapF[i][a];
                    Lf.npar_log2[r] = P.npar_log2[a];
                    for (int q = 0; q < (1 << P.npar_log2[a]); q++) Lf.par[8 * (size_t)r + q] = rmap[i][P.par[8 * (size_t)a + q]];
                }
            }
        }
        rmapF.swap(rmap);
        nmapF.swap(nmap);
    }
    return 0;
}

}  // namespace lbmg
