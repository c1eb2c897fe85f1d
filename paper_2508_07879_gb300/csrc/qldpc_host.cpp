// Host side of the C ABI declared in include/qldpc.h: argument validation, the Tanner-graph
// build (CSR -> check-major slots + per-variable slot lists), device upload, launch-shape choice
// and the end-to-end host-buffer path.  No decoding arithmetic happens here; every step of the
// decoder runs in the sm_103a kernels of msa_kernel.cuh.
#include "qldpc.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include <cuda.h>
#include <cuda_runtime.h>

#include "graph.h"
#include "msa_launch.h"

using namespace qldpc;
using namespace qldpc::detail;

namespace qldpc {

int dc_bucket(int d) { return d <= 8 ? 8 : d <= 16 ? 16 : d <= 32 ? 32 : -1; }
int dv_bucket(int d) { return d <= 4 ? 4 : d <= 8 ? 8 : d <= 16 ? 16 : -1; }
KernelChoice kernel_variant(int dc, int dv, bool uniform, bool latency, bool learned)
{
    if (uniform && dc >= 6 && dc <= 9) return KernelChoice{latency, dc, true, dv_bucket(dv), learned};
    return KernelChoice{latency, dc_bucket(dc), false, dv_bucket(dv), learned};
}

const void *msa_kernel(int precision, const KernelChoice &kc)
{
    if (kc.layered) return msa_kernel_layered(precision, kc);
    if (kc.learned) return msa_kernel_learned(kc);
    if (kc.packed)
        return precision == kINT16 ? msa_kernel_i16x2(kc) : precision == kINT8 ? msa_kernel_i8x2(kc) : msa_kernel_f32x2(kc);
    return precision == kINT16 ? msa_kernel_i16(kc) : precision == kINT8 ? msa_kernel_i8(kc) : msa_kernel_f32(kc);
}

cudaError_t launch_msa(const LaunchParams &p, int precision, const KernelChoice &kc, int threads,
                       int grid_x, size_t smem, cudaStream_t stream)
{
    dim3 grid(unsigned(grid_x), unsigned(p.nprob));
    if (kc.layered) return launch_msa_layered(precision, p, kc, grid, threads, smem, stream);
    if (kc.learned) return launch_msa_learned(p, kc, grid, threads, smem, stream);
    if (kc.packed)
        return precision == kINT16  ? launch_msa_i16x2(p, kc, grid, threads, smem, stream)
               : precision == kINT8 ? launch_msa_i8x2(p, kc, grid, threads, smem, stream)
                                    : launch_msa_f32x2(p, kc, grid, threads, smem, stream);
    return precision == kINT16  ? launch_msa_i16(p, kc, grid, threads, smem, stream)
           : precision == kINT8 ? launch_msa_i8(p, kc, grid, threads, smem, stream)
                                : launch_msa_f32(p, kc, grid, threads, smem, stream);
}

}  // namespace qldpc

namespace {

// ------------------------------------------------------------------------------------------
// Variable lanes.  The variable step runs one thread per variable, so a warp's 32 lanes read and
// write the k-th edge slot of 32 variables at once; slots that share a shared-memory bank (same
// address mod 32 words) serialise.  For a quasi-cyclic code with lift 31 the plain order puts two
// circulant blocks in most warps and costs ~2 wavefronts per access.  The lanes are therefore
// packed per degree class: a warp takes, in order, the first remaining variable whose k-th slots
// all fall in free banks, and is closed early (idle lanes) when none is left, if that pays.
// ------------------------------------------------------------------------------------------
constexpr int kBanks = 32;

// Wavefronts of one warp (or half-warp) access over `banks` banks of one slot word each: the most
// distinct words that fall into one bank.
int warp_wavefronts(const uint32_t *addr, int count, int banks = kBanks)
{
    int dist[kBanks] = {0}, worst = count > 0 ? 1 : 0;
    uint32_t seen[kBanks][kBanks];
    for (int l = 0; l < count; ++l) {
        const int b = int(addr[l] % uint32_t(banks));
        bool dup = false;
        for (int i = 0; i < dist[b]; ++i) dup = dup || seen[b][i] == addr[l];
        if (!dup) seen[b][dist[b]++] = addr[l];
        worst = std::max(worst, dist[b]);
    }
    return worst;
}

// Cost model of one variable-step warp: load and store wavefronts of its edge slots, three for
// Q and gamma, and its instructions (about 8 per edge + 10) at four issues per wavefront cycle.
double lanes_score(const std::vector<int32_t> &lanes, const std::vector<uint32_t> &eaddr,
                   const std::vector<int32_t> &cdeg, int dv)
{
    double s = 0.0;
    uint32_t a[kBanks];
    for (size_t w0 = 0; w0 < lanes.size(); w0 += kBanks) {
        const size_t w1 = std::min(lanes.size(), w0 + kBanks);
        int D = -1;
        for (size_t l = w0; l < w1; ++l)
            if (lanes[l] >= 0) D = std::max(D, cdeg[size_t(lanes[l])]);
        if (D < 0) continue;
        int wf = 0;
        for (int k = 0; k < D; ++k) {
            int c = 0;
            for (size_t l = w0; l < w1; ++l)
                if (lanes[l] >= 0 && k < cdeg[size_t(lanes[l])]) a[c++] = eaddr[size_t(lanes[l]) * dv + k];
            wf += warp_wavefronts(a, c);
        }
        s += 2.0 * wf + 3.0 + (8.0 * D + 10.0) / 4.0;
    }
    return s;
}

// Greedy packing of one candidate; close_at = fewest lanes a warp keeps before it may close early.
std::vector<int32_t> pack_lanes(const std::vector<uint32_t> &order, const std::vector<uint32_t> &eaddr,
                                const std::vector<int32_t> &cdeg, int dv, int close_at)
{
    constexpr size_t kScan = 4096;   // candidates examined per lane
    std::vector<int32_t> lanes;
    lanes.reserve(order.size() + order.size() / 4 + kBanks);
    const size_t n = order.size();
    for (size_t i = 0; i < n;) {
        const int d = cdeg[order[i]];
        size_t j = i;
        while (j < n && cdeg[order[j]] == d) ++j;
        std::vector<char> taken(j - i, 0);
        size_t first = 0, left = j - i;
        while (left > 0) {
            int64_t owner[16][kBanks];   // word held by bank b for the k-th edges, -1 free
            for (int k = 0; k < std::max(d, 1) && k < 16; ++k)
                for (int b = 0; b < kBanks; ++b) owner[k][b] = -1;
            int filled = 0;
            while (filled < kBanks && left > 0) {
                size_t best = SIZE_MAX, scanned = 0;
                int best_cost = 1 << 30;
                for (size_t x = first; x < j - i && scanned < kScan; ++x) {
                    if (taken[x]) continue;
                    ++scanned;
                    const uint32_t v = order[i + x];
                    int c = 0;
                    for (int k = 0; k < d; ++k) {
                        const uint32_t a = eaddr[size_t(v) * dv + k];
                        const int64_t o = owner[k][a % kBanks];
                        c += (o >= 0 && o != int64_t(a)) ? 1 : 0;
                    }
                    if (c < best_cost) {
                        best_cost = c;
                        best = x;
                        if (c == 0) break;
                    }
                }
                if (best_cost > 0 && filled >= close_at) break;
                taken[best] = 1;
                --left;
                const uint32_t v = order[i + best];
                lanes.push_back(int32_t(v));
                for (int k = 0; k < d; ++k) {
                    const uint32_t a = eaddr[size_t(v) * dv + k];
                    if (owner[k][a % kBanks] < 0) owner[k][a % kBanks] = a;
                }
                ++filled;
                while (first < j - i && taken[first]) ++first;
            }
            while (lanes.size() % kBanks) lanes.push_back(-1);
        }
        i = j;
    }
    return lanes;
}

// 8-byte slot words (the paired FP32 messages of the two-shots-per-block kernel) are served a
// half-warp at a time over 16 bank pairs, so there the k-th slots of each half should be distinct
// modulo 16 words.  A warp whose 32 slots are distinct modulo 32 can still put two slots 16 words
// apart in one half.  Which lanes form a half does not change the 4-byte banks (the warp's set of
// slots is the same), so each warp's lanes are reordered by pairwise swaps between its halves while
// a swap lowers the 8-byte wavefronts.
// The 8-byte wavefronts of one warp's k-th slots, idle lanes included: a half with idle lanes
// costs one more unless some bank is free in the whole warp (their scratch slot's 4-byte bank) and
// free in that half modulo 16.
int halves_cost(const int32_t *w, const std::vector<uint32_t> &eaddr, const std::vector<int32_t> &cdeg, int dv, int D)
{
    int c = 0;
    uint32_t a[kBanks];
    for (int k = 0; k < D; ++k) {
        bool used[kBanks] = {false};
        for (int l = 0; l < kBanks; ++l)
            if (w[l] >= 0 && k < cdeg[size_t(w[l])]) used[eaddr[size_t(w[l]) * dv + k] % kBanks] = true;
        for (int h = 0; h < 2; ++h) {
            int cnt = 0;
            bool idle = false, half_used[kBanks / 2] = {false};
            for (int l = h * kBanks / 2; l < (h + 1) * kBanks / 2; ++l) {
                if (w[l] >= 0 && k < cdeg[size_t(w[l])]) {
                    a[cnt] = eaddr[size_t(w[l]) * dv + k];
                    half_used[a[cnt] % (kBanks / 2)] = true;
                    ++cnt;
                } else if (w[l] < 0) {
                    idle = true;
                }
            }
            int wf = warp_wavefronts(a, cnt, kBanks / 2);
            if (idle) {
                bool free_bank = false;
                for (int r = 0; r < kBanks && !free_bank; ++r) free_bank = !used[r] && !half_used[r % (kBanks / 2)];
                wf = free_bank ? std::max(wf, 1) : wf + 1;
            }
            c += wf;
        }
    }
    return c;
}

void split_halves(std::vector<int32_t> &lanes, const std::vector<uint32_t> &eaddr, const std::vector<int32_t> &cdeg,
                  int dv)
{
    for (size_t w0 = 0; w0 + kBanks <= lanes.size(); w0 += kBanks) {
        int32_t *w = lanes.data() + w0;
        int D = -1;
        bool mixed = false;   // a warp that straddles two degree classes keeps its order (degrees stay sorted)
        for (int l = 0; l < kBanks; ++l)
            if (w[l] >= 0) {
                const int d = cdeg[size_t(w[l])];
                mixed = mixed || (D >= 0 && d != D);
                D = std::max(D, d);
            }
        if (mixed || D <= 0) continue;
        int cost = halves_cost(w, eaddr, cdeg, dv, D);
        for (bool improved = true; improved && cost > 2 * D;) {
            improved = false;
            for (int a = 0; a < kBanks / 2; ++a)
                for (int b = kBanks / 2; b < kBanks; ++b) {
                    if (w[a] < 0 && w[b] < 0) continue;
                    std::swap(w[a], w[b]);
                    const int c = halves_cost(w, eaddr, cdeg, dv, D);
                    if (c < cost) {
                        cost = c;
                        improved = true;
                    } else {
                        std::swap(w[a], w[b]);
                    }
                }
        }
    }
}

// The lanes with the lowest cost among the plain degree order and four packings.  A packing may
// add at most an eighth more lanes (plus one warp), so that it never costs a graph its fit in shared
// memory by more than the Q and gamma words of those lanes.
std::vector<int32_t> choose_lanes(const std::vector<uint32_t> &order, const std::vector<uint32_t> &eaddr,
                                  const std::vector<int32_t> &cdeg, int dv)
{
    std::vector<int32_t> best(order.begin(), order.end());
    if (dv > 16) return best;
    double best_s = lanes_score(best, eaddr, cdeg, dv);
    const size_t max_lanes = order.size() + order.size() / 8 + kBanks;
    for (int close_at : {32, 28, 24, 16}) {
        std::vector<int32_t> c = pack_lanes(order, eaddr, cdeg, dv, close_at);
        if (c.size() > max_lanes) continue;
        const double s = lanes_score(c, eaddr, cdeg, dv);
        if (s < best_s) {
            best_s = s;
            best.swap(c);
        }
    }
    return best;
}

// ------------------------------------------------------------------------------------------
// CSR validation and layout (pure host; runs before any CUDA call)
// ------------------------------------------------------------------------------------------
struct HostLayout {
    int32_t dc_max = 0, dv_max = 0;
    bool uniform_rows = true;
    std::vector<uint8_t> rdeg, vdeg;
    std::vector<uint32_t> vslot;   // [dv_max * nv]
    std::vector<uint32_t> vorder;  // [nv] caller's variable of each lane, n for an idle lane
    std::vector<uint32_t> vlane;   // [n] lane of each variable
    std::vector<uint32_t> eslot;   // [nnz] slot j*m + i of CSR edge e
    std::vector<int32_t> slot_edge;// [dc_max * m] CSR edge of each slot, -1 for padding
    std::vector<uint32_t> ecol;    // [dc_max * m] caller's variable of each slot, ~0 for padding
    std::vector<int32_t> layer_ptr;// [nlayers + 1] layered schedule
    std::vector<uint32_t> layer_chk;// [m] checks ordered by (layer, index)
    int32_t max_layer = 0;
    int32_t nv = 0;               // variable lanes (n + idle lanes)
    std::vector<uint16_t> vslot16;// vslot as 16-bit indices (empty when a slot index exceeds 65535)
    std::vector<uint16_t> vchk16; // the check i = slot mod m of each vslot16 entry (same layout)
    std::vector<int32_t> cls_end, cls_deg;   // runs of equal lane degree
    uint32_t m_magic = 0;         // slot / m = umulhi(slot, m_magic) >> m_shift
    int32_t m_shift = 0;
};

int validate_and_layout(const int32_t *row_ptr, const int32_t *col_idx, int32_t m, int32_t n,
                        HostLayout &out)
{
    if (!row_ptr || m <= 0 || n <= 0) return QLDPC_ERR_INVALID_ARG;
    if (row_ptr[0] != 0) return QLDPC_ERR_INVALID_ARG;
    for (int32_t i = 0; i < m; ++i)
        if (row_ptr[i + 1] < row_ptr[i]) return QLDPC_ERR_INVALID_ARG;
    const int64_t nnz = row_ptr[m];
    if (nnz > 0 && !col_idx) return QLDPC_ERR_INVALID_ARG;
    std::vector<int32_t> seen(size_t(n), -1);
    std::vector<int32_t> cdeg(size_t(n), 0);
    int32_t dc_max = 0;
    for (int32_t i = 0; i < m; ++i) {
        const int32_t d = row_ptr[i + 1] - row_ptr[i];
        if (d < 2) return QLDPC_ERR_INVALID_ARG;
        dc_max = std::max(dc_max, d);
        for (int32_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            const int32_t v = col_idx[e];
            if (v < 0 || v >= n) return QLDPC_ERR_INVALID_ARG;
            if (seen[size_t(v)] == i) return QLDPC_ERR_INVALID_ARG;   // repeated column in a row
            seen[size_t(v)] = i;
            cdeg[size_t(v)]++;
        }
    }
    const int32_t dv_max = *std::max_element(cdeg.begin(), cdeg.end());
    if (dc_max > QLDPC_MAX_ROW_DEGREE || dv_max > QLDPC_MAX_COL_DEGREE) return QLDPC_ERR_UNSUPPORTED;
    if (m > QLDPC_MAX_CHECKS) return QLDPC_ERR_UNSUPPORTED;   // (no shot that large fits on chip either)

    out.dc_max = dc_max;
    out.dv_max = dv_max;
    out.rdeg.resize(size_t(m));
    // internal order: descending degree, stable (ties keep the caller's order), then packed into
    // warps of bank-disjoint slots (idle lanes: vorder = n, degree 0)
    std::vector<uint32_t> order(static_cast<size_t>(n));
    for (int32_t v = 0; v < n; ++v) order[size_t(v)] = uint32_t(v);
    std::stable_sort(order.begin(), order.end(), [&](uint32_t a, uint32_t b) { return cdeg[a] > cdeg[b]; });
    const int dv1 = std::max(dv_max, 1);
    std::vector<uint32_t> eaddr(size_t(n) * size_t(dv1), 0u);   // FP32 slot words, ascending checks
    {
        std::vector<int32_t> fill(static_cast<size_t>(n), 0);
        for (int32_t i = 0; i < m; ++i)
            for (int32_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
                const int32_t v = col_idx[e];
                eaddr[size_t(v) * dv1 + size_t(fill[size_t(v)]++)] = uint32_t(e - row_ptr[i]) * uint32_t(m) + uint32_t(i);
            }
    }
    std::vector<int32_t> lanes = choose_lanes(order, eaddr, cdeg, dv1);
    if (lanes.size() % kBanks == 0) split_halves(lanes, eaddr, cdeg, dv1);
    const size_t nv = lanes.size();
    out.nv = int32_t(nv);
    out.vorder.assign(nv, uint32_t(n));
    std::vector<uint32_t> internal(static_cast<size_t>(n), 0u);
    for (size_t u = 0; u < nv; ++u)
        if (lanes[u] >= 0) {
            out.vorder[u] = uint32_t(lanes[u]);
            internal[size_t(lanes[u])] = uint32_t(u);
        }
    out.vlane = internal;
    out.vdeg.assign(nv, 0);
    out.vslot.assign(size_t(dv1) * nv, 0u);
    // Idle lanes: their warp's degree, every edge on a scratch slot dc_max*m + b in a bank the
    // warp's variables leave free for that edge (4-byte words), and where possible one whose bank
    // pair the variables of the lane's half-warp leave free (8-byte words).
    const uint32_t S_words = uint32_t(dc_max) * uint32_t(m);
    for (size_t w0 = 0; w0 < nv; w0 += kBanks) {
        const size_t w1 = std::min(nv, w0 + kBanks);
        int D = 0;
        bool any_idle = false;
        for (size_t l = w0; l < w1; ++l) {
            if (lanes[l] >= 0)
                D = std::max(D, cdeg[size_t(lanes[l])]);
            else
                any_idle = true;
        }
        if (!any_idle) continue;
        for (int k = 0; k < D; ++k) {
            bool used[kBanks] = {false}, used_half[2][kBanks / 2] = {{false}};
            for (size_t l = w0; l < w1; ++l)
                if (lanes[l] >= 0 && k < cdeg[size_t(lanes[l])]) {
                    const uint32_t a = eaddr[size_t(lanes[l]) * dv1 + k];
                    used[a % kBanks] = true;
                    used_half[(l - w0) / (kBanks / 2)][a % (kBanks / 2)] = true;
                }
            for (int h = 0; h < 2; ++h) {
                int b = -1;
                for (int r = 0; r < kBanks && b < 0; ++r)
                    if (!used[r] && !used_half[h][r % (kBanks / 2)]) b = r;
                for (int r = 0; r < kBanks && b < 0; ++r)
                    if (!used[r]) b = r;
                if (b < 0) b = 0;
                const uint32_t sw = (uint32_t(b) + kBanks - S_words % kBanks) % kBanks;   // (S + sw) % 32 == b
                for (size_t l = w0 + size_t(h) * (kBanks / 2); l < std::min(w1, w0 + size_t(h + 1) * (kBanks / 2)); ++l)
                    if (lanes[l] < 0) out.vslot[size_t(k) * nv + l] = S_words + sw;
            }
        }
        for (size_t l = w0; l < w1; ++l)
            if (lanes[l] < 0) out.vdeg[l] = uint8_t(D);
    }
    // Rows are visited in ascending order, so each variable's list is in ascending check order,
    // the order in which the variable step accumulates its sums.
    const size_t S = size_t(dc_max) * size_t(m);
    out.eslot.assign(size_t(nnz), 0u);
    out.slot_edge.assign(S, -1);
    out.ecol.assign(S, ~0u);
    for (int32_t i = 0; i < m; ++i) {
        out.rdeg[size_t(i)] = uint8_t(row_ptr[i + 1] - row_ptr[i]);
        out.uniform_rows = out.uniform_rows && (row_ptr[i + 1] - row_ptr[i]) == dc_max;
        for (int32_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            const uint32_t u = internal[size_t(col_idx[e])];
            const int32_t j = e - row_ptr[i];
            const int32_t k = out.vdeg[u]++;
            out.vslot[size_t(k) * nv + u] = uint32_t(j) * uint32_t(m) + uint32_t(i);
            const size_t sl = size_t(j) * size_t(m) + size_t(i);
            out.eslot[size_t(e)] = uint32_t(sl);
            out.slot_edge[sl] = e;
            out.ecol[sl] = uint32_t(col_idx[e]);
        }
    }
    if (S + size_t(kScratch) <= 65536) {
        out.vslot16.assign(out.vslot.begin(), out.vslot.end());
        out.vchk16.resize(out.vslot.size());
        for (size_t t = 0; t < out.vslot.size(); ++t) out.vchk16[t] = uint16_t(out.vslot[t] % uint32_t(m));
    }
    for (size_t u = 0; u < nv; ++u) {
        if (out.cls_deg.empty() || out.cls_deg.back() != int32_t(out.vdeg[u])) {
            out.cls_end.push_back(int32_t(u));
            out.cls_deg.push_back(int32_t(out.vdeg[u]));
        }
        out.cls_end.back() = int32_t(u) + 1;
    }
    if (out.cls_end.size() > size_t(kMaxDegClasses)) return QLDPC_ERR_UNSUPPORTED;   // degrees are sorted
    // floor(slot / m) for every slot (scratch included) as a multiply-high and a shift: the
    // smallest shift whose rounded-up reciprocal fits 32 bits and divides every slot exactly.
    {
        const uint32_t limit = S_words + uint32_t(kScratch);
        bool found = m == 1;   // one check: every slot belongs to it (the kernels test m == 1)
        for (uint32_t sh = 0; sh < 32 && !found; ++sh) {
            const uint64_t mg = ((uint64_t(1) << (32 + sh)) + uint64_t(m) - 1) / uint64_t(m);
            if (mg >> 32) break;
            bool exact = true;
            for (uint32_t x = 0; x < limit && exact; ++x)
                exact = uint32_t((uint64_t(x) * mg) >> (32 + sh)) == x / uint32_t(m);
            if (exact) {
                out.m_magic = uint32_t(mg);
                out.m_shift = int32_t(sh);
                found = true;
            }
        }
        if (!found) return QLDPC_ERR_UNSUPPORTED;
    }
    // Layered schedule: a check's layer is one more than the largest layer of an earlier check it
    // shares a variable with, so checks of one layer share no variable and every pair of checks
    // that does keeps its ascending order.
    std::vector<int32_t> last(static_cast<size_t>(n), -1), layer(static_cast<size_t>(m), 0);
    int32_t nlayers = 0;
    for (int32_t i = 0; i < m; ++i) {
        int32_t l = 0;
        for (int32_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) l = std::max(l, last[size_t(col_idx[e])] + 1);
        for (int32_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) last[size_t(col_idx[e])] = l;
        layer[size_t(i)] = l;
        nlayers = std::max(nlayers, l + 1);
    }
    out.layer_ptr.assign(size_t(nlayers) + 1, 0);
    for (int32_t i = 0; i < m; ++i) out.layer_ptr[size_t(layer[size_t(i)]) + 1]++;
    for (int32_t l = 0; l < nlayers; ++l) {
        out.max_layer = std::max(out.max_layer, out.layer_ptr[size_t(l) + 1]);
        out.layer_ptr[size_t(l) + 1] += out.layer_ptr[size_t(l)];
    }
    out.layer_chk.assign(size_t(m), 0u);
    std::vector<int32_t> fillp(out.layer_ptr.begin(), out.layer_ptr.end() - 1);
    for (int32_t i = 0; i < m; ++i) out.layer_chk[size_t(fillp[size_t(layer[size_t(i)])]++)] = uint32_t(i);
    return QLDPC_OK;
}

}  // namespace

namespace qldpc {
namespace detail {

bool finite_alpha(float a) { return std::isfinite(a) && a > 0.0f; }

int alpha_fixed(float alpha)   // round_half_away(alpha * 2^15), -1 outside (0, 1]
{
    if (!std::isfinite(alpha) || alpha <= 0.0f || alpha > 1.0f) return -1;
    const int32_t a = int32_t(std::round(alpha * 32768.0f));
    return (a >= 1 && a <= 32768) ? a : -1;
}

int cuda_status(cudaError_t e)
{
    if (e == cudaSuccess) return QLDPC_OK;
    if (e == cudaErrorMemoryAllocation) return QLDPC_ERR_OOM;
    return QLDPC_ERR_CUDA;
}

size_t shot_smem(const qldpc_graph *g, int precision)
{
    return smem_layout(g->m, g->nv, g->dc_max, msg_bytes(precision)).total;
}

// Opt in to more than 48 KB of dynamic shared memory once per kernel variant and size.
// The kernel's own static shared memory counts against the same per-block limit, so a launch
// whose dynamic part fits only without it is refused here (UNSUPPORTED) rather than failing.
int ensure_kernel_attrs(const void *k, size_t smem, size_t smem_optin)
{
    struct Entry {
        const void *k;
        size_t static_bytes, granted;
    };
    static std::mutex mu;
    static std::vector<Entry> known;
    if (!k) return QLDPC_ERR_UNSUPPORTED;
    if (smem > smem_optin) return QLDPC_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(mu);
    Entry *en = nullptr;
    for (auto &x : known)
        if (x.k == k) en = &x;
    if (!en) {
        cudaFuncAttributes fa{};
        cudaError_t e = cudaFuncGetAttributes(&fa, k);
        if (e != cudaSuccess) return cuda_status(e);
        known.push_back(Entry{k, fa.sharedSizeBytes, 0});
        en = &known.back();
    }
    if (smem + en->static_bytes > smem_optin) return QLDPC_ERR_UNSUPPORTED;
    if (smem + en->static_bytes <= 48 * 1024 || en->granted >= smem) return QLDPC_OK;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return cuda_status(e);
    en->granted = smem;
    return QLDPC_OK;
}

// The launch shape of one call.
struct Plan {
    KernelChoice kc{};
    int threads = 0;
    int grid = 0;
    size_t smem = 0;
};

int round32(int x) { return (x + 31) / 32 * 32; }

// Threads per block of the batch kernel: measured within 3 % of the best block size on the
// 192-, 465- and 144-check codes (several small blocks per SM beat few large ones).
constexpr int kBatchThreads = 128;

// Compiled variant for the graphs of one call: exact uniform row degree 6..9, else a bucket.
KernelChoice variant(const qldpc_graph *const *gs, int nprob, bool latency, bool learned)
{
    int dc = 0, dv = 0;
    bool uniform = true;
    for (int i = 0; i < nprob; ++i) {
        dc = std::max(dc, gs[i]->dc_max);
        dv = std::max(dv, gs[i]->dv_max);
        uniform = uniform && gs[i]->uniform_rows && gs[i]->dc_max == gs[0]->dc_max;
    }
    return kernel_variant(dc, dv, uniform, latency, learned);
}

// Resident blocks per SM of a kernel at a block size and shared-memory size.  The runtime's query
// costs host time on the order of the decode itself for small batches, so results are cached.
int blocks_per_sm(const void *k, int threads, size_t smem, int &per_sm)
{
    struct Entry {
        int device;
        const void *k;
        int threads;
        size_t smem;
        int per_sm;
    };
    static std::mutex mu;
    static std::vector<Entry> cache;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return QLDPC_ERR_CUDA;
    {
        std::lock_guard<std::mutex> lk(mu);
        for (const Entry &e : cache)
            if (e.device == dev && e.k == k && e.threads == threads && e.smem == smem) {
                per_sm = e.per_sm;
                return QLDPC_OK;
            }
    }
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, threads, smem);
    if (e != cudaSuccess) return cuda_status(e);
    std::lock_guard<std::mutex> lk(mu);
    cache.push_back(Entry{dev, k, threads, smem, per_sm});
    return QLDPC_OK;
}

int occupancy_grid(const qldpc_graph *g0, const void *k, int threads, size_t smem, int nprob,
                   int32_t batch, int per_sm, int &grid)
{
    if (!per_sm) {
        if (int rc = blocks_per_sm(k, threads, smem, per_sm)) return rc;
        if (per_sm < 1) return QLDPC_ERR_UNSUPPORTED;
    }
    const int64_t slots = std::max<int64_t>(1, int64_t(per_sm) * g0->sm_count / nprob);
    grid = int(std::max<int64_t>(1, std::min<int64_t>(batch, slots)));
    return QLDPC_OK;
}

// Single-shot (latency) path: chosen automatically when every shot of the call gets its own SM,
// or forced with QLDPC_KERNEL_LATENCY.  One pass over the checks and the variables when both fit
// in a block of up to 640 threads, else two passes of a block sized for the larger half.
int plan_latency(const qldpc_graph *const *gs, int nprob, int32_t batch, int precision, bool learned, Plan &pl,
                 bool &chosen)
{
    const qldpc_graph *g0 = gs[0];
    chosen = false;
    if (g0->user_kernel == QLDPC_KERNEL_BATCH || g0->user_kernel == QLDPC_KERNEL_PACKED) return QLDPC_OK;
    const bool forced = g0->user_kernel == QLDPC_KERNEL_LATENCY;
    if (!forced && int64_t(batch) * nprob > g0->sm_count) return QLDPC_OK;
    int one = 32, two = 32;
    size_t smem = 0;
    for (int i = 0; i < nprob; ++i) {
        one = std::max(one, round32(std::max(gs[i]->m, gs[i]->nv)));
        two = std::max(two, round32(std::max((gs[i]->m + 1) / 2, (gs[i]->nv + 1) / 2)));
        smem = std::max(smem, latency_layout(gs[i]->m, gs[i]->dc_max, msg_bytes(precision)).total);
    }
    const int threads = (forced && g0->user_threads) ? g0->user_threads
                                                      : (one <= kLatencyMaxThreads ? one : two);
    bool fits = threads <= kLatencyMaxThreads && smem <= g0->smem_optin;
    for (int i = 0; i < nprob; ++i)
        fits = fits && gs[i]->m <= kLatencyCnPerThread * threads && gs[i]->nv <= kLatencyVnPerThread * threads;
    if (!fits) return forced ? QLDPC_ERR_UNSUPPORTED : QLDPC_OK;
    pl.kc = variant(gs, nprob, true, learned);
    pl.threads = threads;
    pl.smem = smem;
    const void *k = msa_kernel(precision, pl.kc);
    if (int rc = ensure_kernel_attrs(k, smem, g0->smem_optin)) return rc;
    pl.grid = batch;
    if (forced || int64_t(batch) * nprob > g0->sm_count)
        if (int rc = occupancy_grid(g0, k, threads, smem, nprob, batch, g0->user_blocks_per_sm, pl.grid))
            return rc;
    chosen = true;
    return QLDPC_OK;
}

// Throughput path: two shots per block with their messages paired in one slot (every precision,
// unless the graph's launch override asks for one shot per block, or the shot is learned), or one
// shot per block.  Measured on LP-1054 at 65536 shots: FP32 31.7 M/s in pairs against 26.9, INT16
// 31.3 against 25.5, INT8 37.7 (half-precision lanes) against 26.3.
int plan_batch(const qldpc_graph *const *gs, int nprob, int32_t batch, int precision, bool learned, Plan &pl)
{
    const qldpc_graph *g0 = gs[0];
    const int word = precision == QLDPC_FP32 ? 8 : 4;   // bytes of one paired slot
    bool packed = !learned && g0->user_kernel != QLDPC_KERNEL_BATCH;
    for (int i = 0; i < nprob && packed; ++i)
        if (!gs[i]->dg.vslot16) {   // 16-bit slot indices: any graph whose pair of shots fits on chip
            if (g0->user_kernel == QLDPC_KERNEL_PACKED) return QLDPC_ERR_UNSUPPORTED;
            packed = false;
        }
    if (packed && g0->user_kernel != QLDPC_KERNEL_PACKED) {
        // by default only where two shots fit a block's shared memory (beside 1 KB of static shared
        // memory); a graph whose single shot just fits keeps one shot per block
        for (int i = 0; i < nprob; ++i)
            packed = packed && packed_layout(gs[i]->m, gs[i]->nv, gs[i]->dc_max, word).total + 1024 <= g0->smem_optin;
    }
    size_t smem = 0;
    for (int i = 0; i < nprob; ++i)
        smem = std::max(smem, packed ? packed_layout(gs[i]->m, gs[i]->nv, gs[i]->dc_max, word).total
                                     : shot_smem(gs[i], precision));
    pl.kc = variant(gs, nprob, false, learned);
    pl.kc.packed = packed;
    pl.threads = g0->user_threads ? g0->user_threads : kBatchThreads;
    if (packed && pl.threads > kPackedMaxThreads) return QLDPC_ERR_UNSUPPORTED;
    pl.smem = smem;
    const void *k = msa_kernel(precision, pl.kc);
    if (int rc = ensure_kernel_attrs(k, smem, g0->smem_optin)) return rc;
    const int32_t units = packed ? int32_t((int64_t(batch) + 1) / 2) : batch;   // two shots per packed block
    return occupancy_grid(g0, k, pl.threads, smem, nprob, units, g0->user_blocks_per_sm, pl.grid);
}

// Layered schedule: a block per shot with a thread per check of the largest layer (a multiple
// of 32, at most 1024); the grid fills the SMs from occupancy.
int plan_layered(const qldpc_graph *const *gs, int nprob, int32_t batch, int precision, Plan &pl)
{
    const qldpc_graph *g0 = gs[0];
    size_t smem = 0;
    int widest = 1;
    for (int i = 0; i < nprob; ++i) {
        smem = std::max(smem, layered_layout(gs[i]->m, gs[i]->n, gs[i]->dc_max, msg_bytes(precision)).total);
        widest = std::max(widest, gs[i]->dg.max_layer);
    }
    pl.kc = variant(gs, nprob, false, false);
    pl.kc.layered = true;
    pl.threads = std::min(1024, round32(widest));
    // Single-shot regime (every shot gets its own SM), at most 8 layers of rows of degree <= 8 and at
    // most 256 checks per layer: the register-resident kernel (each thread owns one check per layer; Q
    // is the only shared array) has the lower latency.  Batches take the shared-memory kernel, whose
    // smaller register footprint keeps more shots per SM (41.8 against 34.0 M syndromes/s, LP-1054).
    bool reg = pl.threads <= 256 && int64_t(batch) * nprob <= g0->sm_count;
    for (int i = 0; i < nprob; ++i) reg = reg && gs[i]->dg.nlayers <= 8 && gs[i]->dc_max <= 8 && gs[i]->n <= 65536;
    pl.kc.dvb = reg ? 1 : 0;
    if (reg) {
        smem = 0;
        for (int i = 0; i < nprob; ++i) smem = std::max(smem, align16(size_t(gs[i]->n) * 4));
    }
    pl.smem = smem;
    const void *k = msa_kernel(precision, pl.kc);
    if (int rc = ensure_kernel_attrs(k, smem, g0->smem_optin)) return rc;
    return occupancy_grid(g0, k, pl.threads, smem, nprob, batch, 0, pl.grid);
}

int check_device(const qldpc_graph *g)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return QLDPC_ERR_CUDA;
    return dev == g->device ? QLDPC_OK : QLDPC_ERR_INVALID_ARG;
}

// Validate, plan and enqueue one decode.  plan_only: every check and the launch plan of this batch
// (kernel attributes included), but nothing enqueued.
int launch(const qldpc_graph *g0, const qldpc_graph *g1, const Problem *probs, int nprob,
           int32_t batch, int32_t max_iter, float alpha, int32_t precision, uint32_t flags,
           cudaStream_t stream, bool plan_only = false)
{
    if (precision != QLDPC_FP32 && precision != QLDPC_INT16 && precision != QLDPC_INT8) return QLDPC_ERR_INVALID_ARG;
    if ((flags & ~uint32_t(QLDPC_NO_EARLY_STOP | QLDPC_LEARNED | QLDPC_LAYERED)) != 0) return QLDPC_ERR_INVALID_ARG;
    if (batch < 0 || max_iter < 0 || !finite_alpha(alpha)) return QLDPC_ERR_INVALID_ARG;
    const bool learned = (flags & QLDPC_LEARNED) != 0;
    const bool layered = (flags & QLDPC_LAYERED) != 0;
    if (learned && layered) return QLDPC_ERR_INVALID_ARG;
    if (learned) {   // FP32 weights, stop test on, weights set on every graph of the call
        if (precision != QLDPC_FP32 || (flags & QLDPC_NO_EARLY_STOP)) return QLDPC_ERR_INVALID_ARG;
        if (!g0->d_weights || !g1->d_weights) return QLDPC_ERR_INVALID_ARG;
    }
    int aq = 0;
    if (precision == QLDPC_INT16 || precision == QLDPC_INT8) {
        aq = alpha_fixed(alpha);
        if (aq < 0) return QLDPC_ERR_INVALID_ARG;
    }
    if (batch == 0) return QLDPC_OK;

    LaunchParams p{};
    p.nprob = nprob;
    p.batch = batch;
    p.max_iter = max_iter;
    p.alpha = alpha;
    p.alpha_q = aq;
    p.flags = flags & QLDPC_NO_EARLY_STOP;
    for (int i = 0; i < nprob; ++i) p.prob[i] = probs[i];

    // One kernel variant and one block shape serve both problems of a pair.
    const qldpc_graph *gs[2] = {g0, g1};
    cudaStream_t st = stream;
    Plan pl;
    bool latency = false;
    if (layered) {
        if (int rc = plan_layered(gs, nprob, batch, precision, pl)) return rc;
    } else {
        if (int rc = plan_latency(gs, nprob, batch, precision, learned, pl, latency)) return rc;
        if (!latency)
            if (int rc = plan_batch(gs, nprob, batch, precision, learned, pl)) return rc;
    }
    if (plan_only) return QLDPC_OK;
    if (!latency && (pl.kc.packed || pl.grid < batch)) {
        // more shots than blocks (or the packed kernel, whose lanes always take shots from a counter):
        // claim them dynamically from a zeroed counter pair of the ring
        p.next_shot = g0->d_counters + 2 * size_t(g0->counter_seq.fetch_add(1) % kShotCounterSlots);
        if (cudaError_t e = cudaMemsetAsync(p.next_shot, 0, 2 * sizeof(int32_t), st)) return cuda_status(e);
    }
    return cuda_status(launch_msa(p, precision, pl.kc, pl.threads, pl.grid, pl.smem, st));
}

Problem make_problem(const qldpc_graph *g, const uint8_t *syn, const float *prior, uint8_t *err,
                     int32_t *iters, uint8_t *ok, float *post)
{
    Problem pr{};
    pr.g = g->dg;
    pr.syn = syn;
    pr.prior = prior;
    pr.err = err;
    pr.iters = iters;
    pr.ok = ok;
    pr.post = post;
    pr.weights = g->d_weights;
    pr.learned_iters = g->learned_T;
    return pr;
}

int decode_plan(const qldpc_graph *g, int32_t batch, int32_t max_iter, float alpha, int32_t precision,
                uint32_t flags)
{
    if (!g || batch < 0) return QLDPC_ERR_INVALID_ARG;
    if (int rc = check_device(g)) return rc;
    const Problem pr = make_problem(g, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr);
    return launch(g, g, &pr, 1, batch, max_iter, alpha, precision, flags, nullptr, true);
}

void free_stage(qldpc_graph *g)
{
    if (g->d_stage) cudaFree(g->d_stage);
    if (g->h_stage) cudaFreeHost(g->h_stage);
    g->d_stage = nullptr;
    g->h_stage = nullptr;
    g->h_stage_bytes = 0;
    g->d_syn = g->d_err = g->d_ok = nullptr;
    g->d_iters = nullptr;
    g->d_prior = nullptr;
    g->cap = 0;
}

constexpr size_t kHostStageMax = 64 * 1024;   // outputs up to this size return in one copy

int reserve_stage(qldpc_graph *g, int32_t max_batch)
{
    if (max_batch <= g->cap && g->d_prior) return QLDPC_OK;
    const int32_t cap = std::max(max_batch, g->cap);
    const size_t syn_b = align16(size_t(cap) * g->m);
    const size_t err_b = align16(size_t(cap) * g->n);
    const size_t it_b = align16(size_t(cap) * 4);
    const size_t ok_b = align16(size_t(cap));
    const size_t pr_b = align16(size_t(g->n) * 4);
    void *blk = nullptr;
    cudaError_t e = cudaMalloc(&blk, syn_b + err_b + it_b + ok_b + pr_b);
    if (e != cudaSuccess) return cuda_status(e);
    void *hblk = nullptr;
    const size_t h_b = std::min(err_b + it_b + ok_b, kHostStageMax);
    e = cudaMallocHost(&hblk, h_b);
    if (e != cudaSuccess) {
        cudaFree(blk);
        return cuda_status(e);
    }
    free_stage(g);
    char *b = static_cast<char *>(blk);
    g->d_stage = blk;
    g->d_syn = reinterpret_cast<uint8_t *>(b);
    g->d_err = reinterpret_cast<uint8_t *>(b + syn_b);
    g->d_iters = reinterpret_cast<int32_t *>(b + syn_b + err_b);
    g->d_ok = reinterpret_cast<uint8_t *>(b + syn_b + err_b + it_b);
    g->d_prior = reinterpret_cast<float *>(b + syn_b + err_b + it_b + ok_b);
    g->h_stage = static_cast<uint8_t *>(hblk);
    g->h_stage_bytes = h_b;
    g->prior_valid = false;
    g->cap = cap;
    return QLDPC_OK;
}

// Device-accessible address of [p, p + bytes) when the whole range lies in ONE page-locked host
// allocation known to CUDA (cudaHostAlloc / cudaMallocHost / cudaHostRegister), else nullptr.
// The extent comes from the driver's allocation range, so a buffer that merely starts in pinned
// memory is never read or written by a kernel beyond that allocation.
using PointerAttrFn = CUresult (*)(void *, CUpointer_attribute, CUdeviceptr);

PointerAttrFn pointer_attr_fn()
{
    static PointerAttrFn fn = [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuPointerGetAttribute", &f, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            f = nullptr;
        return reinterpret_cast<PointerAttrFn>(f);
    }();
    return fn;
}

void *mapped_host_range(const void *p, size_t bytes)
{
    if (!p || bytes == 0) return nullptr;
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type != cudaMemoryTypeHost || !a.devicePointer) return nullptr;
    PointerAttrFn fn = pointer_attr_fn();
    if (!fn) return nullptr;
    CUdeviceptr start = 0;
    size_t size = 0;
    const CUdeviceptr dp = reinterpret_cast<CUdeviceptr>(a.devicePointer);
    if (fn(&start, CU_POINTER_ATTRIBUTE_RANGE_START_ADDR, dp) != CUDA_SUCCESS) return nullptr;
    if (fn(&size, CU_POINTER_ATTRIBUTE_RANGE_SIZE, dp) != CUDA_SUCCESS) return nullptr;
    if (start == 0 || size == 0 || dp < start || dp - start + bytes > size) return nullptr;
    return a.devicePointer;
}

// The graph's device copy of the prior, uploaded only when it differs from the last one (caller
// holds host_mu and has reserved the staging).
int upload_prior(qldpc_graph *g, const float *h_prior, cudaStream_t st)
{
    const size_t prior_b = size_t(g->n) * sizeof(float);
    if (g->prior_valid && std::memcmp(g->prior_cache.data(), h_prior, prior_b) == 0) return QLDPC_OK;
    g->prior_cache.assign(h_prior, h_prior + g->n);
    const cudaError_t e = cudaMemcpyAsync(g->d_prior, g->prior_cache.data(), prior_b, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_status(e);
    g->prior_valid = true;
    return QLDPC_OK;
}

}  // namespace detail
}  // namespace qldpc

extern "C" {

int qldpc_graph_create(const int32_t *row_ptr, const int32_t *col_idx, int32_t m, int32_t n,
                       qldpc_graph **out)
{
    if (!out) return QLDPC_ERR_INVALID_ARG;
    *out = nullptr;
    HostLayout hl;
    int rc = validate_and_layout(row_ptr, col_idx, m, n, hl);
    if (rc) return rc;

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return QLDPC_ERR_CUDA;
    cudaDeviceProp prop{};
    e = cudaGetDeviceProperties(&prop, dev);
    if (e != cudaSuccess) return QLDPC_ERR_CUDA;

    qldpc_graph *g = new (std::nothrow) qldpc_graph();
    if (!g) return QLDPC_ERR_OOM;
    g->device = dev;
    g->sm_count = prop.multiProcessorCount;
    g->smem_optin = prop.sharedMemPerBlockOptin;
    g->m = m;
    g->n = n;
    g->nv = hl.nv;
    g->nnz = row_ptr[m];
    g->dc_max = hl.dc_max;
    g->dv_max = hl.dv_max;
    g->uniform_rows = hl.uniform_rows;
    // The FP32 working set is the larger one; reject graphs whose shot does not fit on chip.
    if (shot_smem(g, QLDPC_FP32) > g->smem_optin && shot_smem(g, QLDPC_INT16) > g->smem_optin) {
        delete g;
        return QLDPC_ERR_UNSUPPORTED;
    }

    // one device block: vslot | vdeg | rdeg | vperm | eslot | slot_edge | ecol | layer_ptr | layer_chk |
    // shot counters | vslot16 | vlane | vchk16
    constexpr int kArrays = 13;
    const size_t sizes[kArrays] = {hl.vslot.size() * sizeof(uint32_t), size_t(hl.nv), size_t(m),
                                   size_t(hl.nv) * sizeof(uint32_t), hl.eslot.size() * sizeof(uint32_t),
                                   hl.slot_edge.size() * sizeof(int32_t), hl.ecol.size() * sizeof(uint32_t),
                                   hl.layer_ptr.size() * sizeof(int32_t), hl.layer_chk.size() * sizeof(uint32_t),
                                   size_t(kShotCounterSlots) * 2 * sizeof(int32_t),
                                   hl.vslot16.size() * sizeof(uint16_t), hl.vlane.size() * sizeof(uint32_t),
                                   hl.vchk16.size() * sizeof(uint16_t)};
    const void *srcs[kArrays] = {hl.vslot.data(), hl.vdeg.data(), hl.rdeg.data(), hl.vorder.data(),
                                 hl.eslot.data(), hl.slot_edge.data(), hl.ecol.data(),
                                 hl.layer_ptr.data(), hl.layer_chk.data(), nullptr, hl.vslot16.data(),
                                 hl.vlane.data(), hl.vchk16.data()};
    size_t offs[kArrays], total = 0;
    for (int i = 0; i < kArrays; ++i) {
        offs[i] = total;
        total += align16(std::max<size_t>(sizes[i], 1));
    }
    e = cudaMalloc(&g->d_block, total);
    if (e != cudaSuccess) {
        delete g;
        return cuda_status(e);
    }
    char *b = static_cast<char *>(g->d_block);
    for (int i = 0; i < kArrays && e == cudaSuccess; ++i)
        if (sizes[i] && srcs[i]) e = cudaMemcpy(b + offs[i], srcs[i], sizes[i], cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(g->d_block);
        delete g;
        return cuda_status(e);
    }
    g->dg.vslot = reinterpret_cast<const uint32_t *>(b + offs[0]);
    g->dg.vdeg = reinterpret_cast<const uint8_t *>(b + offs[1]);
    g->dg.rdeg = reinterpret_cast<const uint8_t *>(b + offs[2]);
    g->dg.vperm = reinterpret_cast<const uint32_t *>(b + offs[3]);
    g->dg.eslot = reinterpret_cast<const uint32_t *>(b + offs[4]);
    g->dg.slot_edge = reinterpret_cast<const int32_t *>(b + offs[5]);
    g->dg.ecol = reinterpret_cast<const uint32_t *>(b + offs[6]);
    g->dg.layer_ptr = reinterpret_cast<const int32_t *>(b + offs[7]);
    g->dg.layer_chk = reinterpret_cast<const uint32_t *>(b + offs[8]);
    g->d_counters = reinterpret_cast<int32_t *>(b + offs[9]);
    g->dg.nlayers = int32_t(hl.layer_ptr.size()) - 1;
    g->dg.max_layer = hl.max_layer;
    g->dg.nnz = g->nnz;
    g->dg.m = m;
    g->dg.n = n;
    g->dg.nv = hl.nv;
    g->dg.m_magic = hl.m_magic;
    g->dg.m_shift = hl.m_shift;
    g->dg.dc_max = hl.dc_max;
    g->dg.dv_max = hl.dv_max;
    g->dg.vslot16 = hl.vslot16.empty() ? nullptr : reinterpret_cast<const uint16_t *>(b + offs[10]);
    g->dg.vlane = reinterpret_cast<const uint32_t *>(b + offs[11]);
    g->dg.vchk16 = hl.vchk16.empty() ? nullptr : reinterpret_cast<const uint16_t *>(b + offs[12]);
    g->dg.ncls = int32_t(hl.cls_end.size());
    for (size_t c = 0; c < hl.cls_end.size(); ++c) {
        g->dg.cls_end[c] = hl.cls_end[c];
        g->dg.cls_deg[c] = hl.cls_deg[c];
    }
    *out = g;
    return QLDPC_OK;
}

int qldpc_graph_create_csc(const int32_t *col_ptr, const int32_t *row_idx, int32_t m, int32_t n,
                           qldpc_graph **out)
{
    if (!out) return QLDPC_ERR_INVALID_ARG;
    *out = nullptr;
    if (!col_ptr || m <= 0 || n <= 0 || col_ptr[0] != 0) return QLDPC_ERR_INVALID_ARG;
    for (int32_t v = 0; v < n; ++v)
        if (col_ptr[v + 1] < col_ptr[v]) return QLDPC_ERR_INVALID_ARG;
    const int32_t nnz = col_ptr[n];
    if (nnz > 0 && !row_idx) return QLDPC_ERR_INVALID_ARG;
    std::vector<int32_t> row_ptr(size_t(m) + 1, 0);
    std::vector<int32_t> col(static_cast<size_t>(nnz));
    for (int32_t e = 0; e < nnz; ++e) {
        const int32_t r = row_idx[e];
        if (r < 0 || r >= m) return QLDPC_ERR_INVALID_ARG;
        row_ptr[size_t(r) + 1]++;
    }
    for (int32_t i = 0; i < m; ++i) row_ptr[size_t(i) + 1] += row_ptr[size_t(i)];
    std::vector<int32_t> fill(row_ptr.begin(), row_ptr.end() - 1);
    for (int32_t v = 0; v < n; ++v)
        for (int32_t e = col_ptr[v]; e < col_ptr[v + 1]; ++e) col[size_t(fill[size_t(row_idx[e])]++)] = v;
    return qldpc_graph_create(row_ptr.data(), col.data(), m, n, out);
}

void qldpc_graph_destroy(qldpc_graph *g)
{
    if (!g) return;
    free_stage(g);
    if (g->d_block) cudaFree(g->d_block);
    if (g->d_weights) cudaFree(g->d_weights);
    delete g;
}

int qldpc_graph_dims(const qldpc_graph *g, int32_t *m, int32_t *n, int32_t *nnz,
                     int32_t *max_row_degree, int32_t *max_col_degree)
{
    if (!g) return QLDPC_ERR_INVALID_ARG;
    if (m) *m = g->m;
    if (n) *n = g->n;
    if (nnz) *nnz = g->nnz;
    if (max_row_degree) *max_row_degree = g->dc_max;
    if (max_col_degree) *max_col_degree = g->dv_max;
    return QLDPC_OK;
}

int qldpc_graph_layers(const qldpc_graph *g, int32_t *layers, int32_t *widest)
{
    if (!g) return QLDPC_ERR_INVALID_ARG;
    if (layers) *layers = g->dg.nlayers;
    if (widest) *widest = g->dg.max_layer;
    return QLDPC_OK;
}

int qldpc_graph_footprint(const qldpc_graph *g, int32_t precision, int32_t *lanes, size_t *shot_bytes)
{
    if (!g) return QLDPC_ERR_INVALID_ARG;
    if (precision != QLDPC_FP32 && precision != QLDPC_INT16 && precision != QLDPC_INT8) return QLDPC_ERR_INVALID_ARG;
    if (lanes) *lanes = g->nv;
    if (shot_bytes) *shot_bytes = shot_smem(g, precision);
    return QLDPC_OK;
}

int qldpc_graph_set_launch(qldpc_graph *g, int32_t kernel, int32_t threads_per_block,
                           int32_t blocks_per_sm)
{
    if (!g) return QLDPC_ERR_INVALID_ARG;
    if (kernel != QLDPC_KERNEL_AUTO && kernel != QLDPC_KERNEL_BATCH && kernel != QLDPC_KERNEL_LATENCY &&
        kernel != QLDPC_KERNEL_PACKED)
        return QLDPC_ERR_INVALID_ARG;
    if (threads_per_block != 0 && (threads_per_block < 32 || threads_per_block > 1024 || threads_per_block % 32))
        return QLDPC_ERR_INVALID_ARG;
    if (blocks_per_sm < 0 || blocks_per_sm > 32) return QLDPC_ERR_INVALID_ARG;
    if (kernel == QLDPC_KERNEL_AUTO && (threads_per_block || blocks_per_sm)) return QLDPC_ERR_INVALID_ARG;
    if (int rc = check_device(g)) return rc;
    const int saved[3] = {g->user_kernel, g->user_threads, g->user_blocks_per_sm};
    g->user_kernel = kernel;
    g->user_threads = threads_per_block;
    g->user_blocks_per_sm = 0;
    // the shape must be launchable, and the requested residency achievable, in both precisions
    const qldpc_graph *gs[1] = {g};
    int rc = QLDPC_OK;
    for (int prec : {QLDPC_FP32, QLDPC_INT16, QLDPC_INT8}) {
        Plan pl;
        bool latency = false;
        const int32_t big = int32_t(1) << 30;
        rc = plan_latency(gs, 1, big, prec, false, pl, latency);
        if (rc == QLDPC_OK && !latency) rc = plan_batch(gs, 1, big, prec, false, pl);
        if (rc == QLDPC_OK && blocks_per_sm && pl.grid < blocks_per_sm * g->sm_count) rc = QLDPC_ERR_UNSUPPORTED;
        if (rc) break;
    }
    if (rc) {
        g->user_kernel = saved[0];
        g->user_threads = saved[1];
        g->user_blocks_per_sm = saved[2];
        return rc;
    }
    g->user_blocks_per_sm = blocks_per_sm;
    return QLDPC_OK;
}

int qldpc_graph_reserve(qldpc_graph *g, int32_t max_batch)
{
    if (!g || max_batch < 0) return QLDPC_ERR_INVALID_ARG;
    if (int rc = check_device(g)) return rc;
    std::lock_guard<std::mutex> lk(g->host_mu);
    return reserve_stage(g, std::max(max_batch, 1));
}

int qldpc_decode_ex(const qldpc_graph *g, const uint8_t *syndromes, int32_t batch,
                    const float *prior_llr, int32_t max_iter, float alpha, uint8_t *out_err,
                    int32_t *out_iters, uint8_t *out_ok, float *out_post, int32_t precision,
                    uint32_t flags, void *stream)
{
    if (!g) return QLDPC_ERR_INVALID_ARG;
    if (batch > 0 && (!syndromes || !prior_llr || !out_err || !out_iters || !out_ok))
        return QLDPC_ERR_INVALID_ARG;
    if (int rc = check_device(g)) return rc;
    const Problem pr = make_problem(g, syndromes, prior_llr, out_err, out_iters, out_ok, out_post);
    return launch(g, g, &pr, 1, batch, max_iter, alpha, precision, flags,
                  static_cast<cudaStream_t>(stream));
}

int qldpc_decode(const qldpc_graph *g, const uint8_t *syndromes, int32_t batch,
                 const float *prior_llr, int32_t max_iter, float alpha, uint8_t *out_err,
                 int32_t *out_iters, uint8_t *out_ok)
{
    return qldpc_decode_ex(g, syndromes, batch, prior_llr, max_iter, alpha, out_err, out_iters,
                           out_ok, nullptr, QLDPC_FP32, 0u, nullptr);
}

int qldpc_decode_pair(const qldpc_graph *g_z, const qldpc_graph *g_x, const uint8_t *s_x,
                      const uint8_t *s_z, int32_t batch, const float *prior_x, const float *prior_z,
                      int32_t max_iter, float alpha, uint8_t *err_x, uint8_t *err_z,
                      int32_t *iters_x, int32_t *iters_z, uint8_t *ok_x, uint8_t *ok_z,
                      float *post_x, float *post_z, int32_t precision, uint32_t flags, void *stream)
{
    if (!g_z || !g_x) return QLDPC_ERR_INVALID_ARG;
    if (g_z->n != g_x->n || g_z->device != g_x->device) return QLDPC_ERR_INVALID_ARG;
    if (batch > 0 && (!s_x || !s_z || !prior_x || !prior_z || !err_x || !err_z || !iters_x ||
                      !iters_z || !ok_x || !ok_z))
        return QLDPC_ERR_INVALID_ARG;
    if (int rc = check_device(g_z)) return rc;
    const Problem pr[2] = {make_problem(g_z, s_x, prior_x, err_x, iters_x, ok_x, post_x),
                           make_problem(g_x, s_z, prior_z, err_z, iters_z, ok_z, post_z)};
    return launch(g_z, g_x, pr, 2, batch, max_iter, alpha, precision, flags,
                  static_cast<cudaStream_t>(stream));
}

int qldpc_decode_host(qldpc_graph *g, const uint8_t *h_syndromes, int32_t batch,
                      const float *h_prior, int32_t max_iter, float alpha, uint8_t *h_err,
                      int32_t *h_iters, uint8_t *h_ok, int32_t precision, uint32_t flags,
                      void *stream)
{
    if (!g) return QLDPC_ERR_INVALID_ARG;
    if (batch < 0) return QLDPC_ERR_INVALID_ARG;
    if (batch > 0 && (!h_syndromes || !h_prior || !h_err || !h_iters || !h_ok))
        return QLDPC_ERR_INVALID_ARG;
    if (int rc = check_device(g)) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // every argument check of the decode itself, before anything is enqueued
    if (int rc = launch(g, g, nullptr, 1, 0, max_iter, alpha, precision, flags, st)) return rc;
    if (batch == 0) return QLDPC_OK;
    std::lock_guard<std::mutex> lk(g->host_mu);
    if (int rc = reserve_stage(g, batch)) return rc;
    cudaError_t e = cudaSuccess;
    // Page-locked buffers: the kernel reads the syndromes and writes the results in host memory
    // directly (NVLink-C2C on Grace-Blackwell), so the call is one launch and one synchronize.
    void *z_syn = mapped_host_range(h_syndromes, size_t(batch) * g->m);
    void *z_err = z_syn ? mapped_host_range(h_err, size_t(batch) * g->n) : nullptr;
    void *z_it = z_err ? mapped_host_range(h_iters, size_t(batch) * 4) : nullptr;
    void *z_ok = z_it ? mapped_host_range(h_ok, size_t(batch)) : nullptr;
    if (int rc = upload_prior(g, h_prior, st)) return rc;
    if (z_ok) {
        const Problem pz = make_problem(g, static_cast<const uint8_t *>(z_syn), g->d_prior,
                                        static_cast<uint8_t *>(z_err), static_cast<int32_t *>(z_it),
                                        static_cast<uint8_t *>(z_ok), nullptr);
        int rc = launch(g, g, &pz, 1, batch, max_iter, alpha, precision, flags, st);
        const cudaError_t se = cudaStreamSynchronize(st);
        if (rc) return rc;
        return cuda_status(se);
    }
    e = cudaMemcpyAsync(g->d_syn, h_syndromes, size_t(batch) * g->m, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_status(e);
    const Problem pr = make_problem(g, g->d_syn, g->d_prior, g->d_err, g->d_iters, g->d_ok, nullptr);
    int rc = launch(g, g, &pr, 1, batch, max_iter, alpha, precision, flags, st);
    if (rc) {
        cudaStreamSynchronize(st);
        return rc;
    }
    // e_hat, iterations and ok are contiguous in the staging: a small batch comes back in one
    // copy through page-locked staging, a large one straight into the caller's buffers.
    const size_t err_b = size_t(batch) * g->n;
    const size_t out_b = size_t(g->d_ok - g->d_err) + size_t(batch);
    if (g->h_stage && out_b <= g->h_stage_bytes) {
        e = cudaMemcpyAsync(g->h_stage, g->d_err, out_b, cudaMemcpyDeviceToHost, st);
        const cudaError_t se = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_status(e);
        if (se != cudaSuccess) return cuda_status(se);
        std::memcpy(h_err, g->h_stage, err_b);
        std::memcpy(h_iters, g->h_stage + (reinterpret_cast<uint8_t *>(g->d_iters) - g->d_err), size_t(batch) * 4);
        std::memcpy(h_ok, g->h_stage + (g->d_ok - g->d_err), size_t(batch));
        return QLDPC_OK;
    }
    e = cudaMemcpyAsync(h_err, g->d_err, err_b, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h_iters, g->d_iters, size_t(batch) * 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_ok, g->d_ok, size_t(batch), cudaMemcpyDeviceToHost, st);
    const cudaError_t se = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_status(e);
    return cuda_status(se);
}

int qldpc_decode_pair_host(qldpc_graph *g_z, qldpc_graph *g_x, const uint8_t *h_sx, const uint8_t *h_sz,
                           int32_t batch, const float *h_prior_x, const float *h_prior_z, int32_t max_iter,
                           float alpha, uint8_t *h_err_x, uint8_t *h_err_z, int32_t *h_iters_x,
                           int32_t *h_iters_z, uint8_t *h_ok_x, uint8_t *h_ok_z, int32_t precision,
                           uint32_t flags, void *stream)
{
    if (!g_z || !g_x || g_z == g_x || batch < 0) return QLDPC_ERR_INVALID_ARG;
    if (g_z->n != g_x->n || g_z->device != g_x->device) return QLDPC_ERR_INVALID_ARG;
    if (batch > 0 && (!h_sx || !h_sz || !h_prior_x || !h_prior_z || !h_err_x || !h_err_z || !h_iters_x ||
                      !h_iters_z || !h_ok_x || !h_ok_z))
        return QLDPC_ERR_INVALID_ARG;
    if (int rc = check_device(g_z)) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Problem pr[2] = {make_problem(g_z, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr),
                     make_problem(g_x, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr)};
    // every argument check and the launch plan, before anything is enqueued
    if (int rc = launch(g_z, g_x, pr, 2, batch, max_iter, alpha, precision, flags, st, true)) return rc;
    if (batch == 0) return QLDPC_OK;
    std::scoped_lock lk(g_z->host_mu, g_x->host_mu);
    if (int rc = reserve_stage(g_z, batch)) return rc;
    if (int rc = reserve_stage(g_x, batch)) return rc;
    if (int rc = upload_prior(g_z, h_prior_x, st)) return rc;
    if (int rc = upload_prior(g_x, h_prior_z, st)) return rc;
    // Page-locked buffers: the kernel reads the syndromes and writes the results in host memory.
    const size_t bx = size_t(batch) * g_z->m, bz = size_t(batch) * g_x->m, be = size_t(batch) * g_z->n;
    void *z[8] = {mapped_host_range(h_sx, bx), mapped_host_range(h_sz, bz), mapped_host_range(h_err_x, be),
                  mapped_host_range(h_err_z, be), mapped_host_range(h_iters_x, size_t(batch) * 4),
                  mapped_host_range(h_iters_z, size_t(batch) * 4), mapped_host_range(h_ok_x, size_t(batch)),
                  mapped_host_range(h_ok_z, size_t(batch))};
    bool zero_copy = true;
    for (void *x : z) zero_copy = zero_copy && x;
    if (zero_copy) {
        pr[0] = make_problem(g_z, static_cast<const uint8_t *>(z[0]), g_z->d_prior, static_cast<uint8_t *>(z[2]),
                             static_cast<int32_t *>(z[4]), static_cast<uint8_t *>(z[6]), nullptr);
        pr[1] = make_problem(g_x, static_cast<const uint8_t *>(z[1]), g_x->d_prior, static_cast<uint8_t *>(z[3]),
                             static_cast<int32_t *>(z[5]), static_cast<uint8_t *>(z[7]), nullptr);
        const int rc = launch(g_z, g_x, pr, 2, batch, max_iter, alpha, precision, flags, st);
        const cudaError_t se = cudaStreamSynchronize(st);
        if (rc) return rc;
        return cuda_status(se);
    }
    cudaError_t e = cudaMemcpyAsync(g_z->d_syn, h_sx, bx, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(g_x->d_syn, h_sz, bz, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) {
        cudaStreamSynchronize(st);
        return cuda_status(e);
    }
    pr[0] = make_problem(g_z, g_z->d_syn, g_z->d_prior, g_z->d_err, g_z->d_iters, g_z->d_ok, nullptr);
    pr[1] = make_problem(g_x, g_x->d_syn, g_x->d_prior, g_x->d_err, g_x->d_iters, g_x->d_ok, nullptr);
    if (int rc = launch(g_z, g_x, pr, 2, batch, max_iter, alpha, precision, flags, st)) {
        cudaStreamSynchronize(st);
        return rc;
    }
    const qldpc_graph *gs[2] = {g_z, g_x};
    uint8_t *errs[2] = {h_err_x, h_err_z}, *oks[2] = {h_ok_x, h_ok_z};
    int32_t *its[2] = {h_iters_x, h_iters_z};
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
        e = cudaMemcpyAsync(errs[i], gs[i]->d_err, be, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(its[i], gs[i]->d_iters, size_t(batch) * 4, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(oks[i], gs[i]->d_ok, size_t(batch), cudaMemcpyDeviceToHost, st);
    }
    const cudaError_t se = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_status(e);
    return cuda_status(se);
}

const char *qldpc_status_string(int status)
{
    switch (status) {
    case QLDPC_OK: return "QLDPC_OK";
    case QLDPC_PENDING: return "QLDPC_PENDING: the request is still running";
    case QLDPC_BUSY: return "QLDPC_BUSY: the ring is full";
    case QLDPC_ERR_INVALID_ARG: return "QLDPC_ERR_INVALID_ARG: invalid argument";
    case QLDPC_ERR_UNSUPPORTED: return "QLDPC_ERR_UNSUPPORTED: graph exceeds a kernel limit";
    case QLDPC_ERR_OOM: return "QLDPC_ERR_OOM: out of memory";
    case QLDPC_ERR_CUDA: return "QLDPC_ERR_CUDA: CUDA runtime error";
    case QLDPC_ERR_TIMEOUT: return "QLDPC_ERR_TIMEOUT: device-side wait expired";
    default: return "unknown qldpc status";
    }
}

}  // extern "C"
