// C ABI of the GNN-MPC library: handles, workspace layout, and the order of
// the kernels of one real-time iteration (Algorithm 1).
#include <algorithm>
#include <atomic>
#include <cstring>
#include <numeric>

#include "admm.h"
#include "ctx.h"
#include "kernels.h"

namespace gmi {

static thread_local std::string g_err;
static std::atomic<unsigned long long> g_launches{0};

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

void set_error(const char* fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
}
void clear_error() { g_err.clear(); }

// ---------------------------------------------------------------- reverse-mode cones
// For every seed (output node) s: the nodes reaching s in at most r edges (BFS
// over predecessors), and the edges into them.  See struct Cones.
static int row_of(const std::vector<int>& node, const std::vector<int>& ptr, int s, int n) {
    auto b = node.begin() + ptr[s], e = node.begin() + ptr[s + 1];
    auto it = std::lower_bound(b, e, n);
    return (it != e && *it == n) ? (int)(it - node.begin()) : -1;
}

// Supports of the forward-mode sensitivity columns (matrix-free condensing, struct Tangents).
// Row contexts of the tangent launches (struct Tangents): per (stage k, layer l), tangent t =
// i nu + a, the support's positions p in actuator a's hop order.  The row of node n (edge q) in a
// layer with radius R is that layer's offset of t plus n's (q's) position, if the position lies
// within the first count(a, R) of the order, else -1.
static void build_tangent_ctx(const gm_graph& g, int K, int N, Tangents& T) {
    const int M = g.M, E = g.E, nu = g.nu, R1 = T.Rmax + 1, L = N * nu + 1;
    auto ncount = [&](int a, int R) { return R < 0 ? 0 : T.ncnt[(size_t)a * R1 + std::min(R, T.Rmax)]; };
    auto ecount = [&](int a, int R) { return R < 0 ? 0 : T.ecnt[(size_t)a * R1 + std::min(R, T.Rmax)]; };
    T.nbase.assign((size_t)N * (K + 1), 0);
    T.ebase.assign((size_t)N * (K + 1), 0);
    long nb = 0, eb = 0;
    for (int k = 0; k < N; ++k)
        for (int l = 0; l <= K; ++l) {
            const size_t kl = (size_t)k * (K + 1) + l, base = kl * L;
            T.nbase[kl] = nb;
            T.ebase[kl] = eb;
            nb += T.noff[base + (k + 1) * nu];
            eb += T.eoff[base + (k + 1) * nu];
        }
    T.nctx.assign((size_t)4 * nb, -1);
    T.ectx.assign((size_t)4 * eb, -1);
    T.aptr.assign((size_t)nb + 1, 0);
    T.alist.clear();
    for (int k = 0; k < N; ++k)
        for (int l = 0; l <= K; ++l) {
            const size_t kl = (size_t)k * (K + 1) + l, base = kl * L, pbase = base - (size_t)L;   // layer l - 1
            for (int t = 0; t < (k + 1) * nu; ++t) {
                const int i = t / nu, a = t % nu, r0 = K * (k - i);
                // node rows of layer l (radius r0 + l)
                int* nc = T.nctx.data() + 4 * (T.nbase[kl] + T.noff[base + t]);
                const int nn = T.noff[base + t + 1] - T.noff[base + t];
                const int nprev = l > 0 ? ncount(a, r0 + l - 1) : 0;
                const int ecnt_l = l > 0 ? ecount(a, r0 + l - 1) : 0;   // edge layer l (message sum)
                for (int p = 0; p < nn; ++p) {
                    const int n = T.norder[(size_t)a * M + p];
                    nc[4 * p] = p < nprev ? T.noff[pbase + t] + p : -1;
                    nc[4 * p + 1] = t;
                    nc[4 * p + 2] = n;
                    nc[4 * p + 3] = i < k ? 1 : 0;
                    T.aptr[(size_t)(T.nbase[kl] + T.noff[base + t] + p)] = (int)T.alist.size();
                    if (l > 0)
                        for (int q = g.in_ptr[n]; q < g.in_ptr[n + 1]; ++q) {
                            const int pe = T.epos[(size_t)a * E + q];
                            if (pe < ecnt_l) T.alist.push_back(T.eoff[base + t] + pe);
                        }
                }
                if (E == 0) continue;
                // edge rows of layer l
                int* ec = T.ectx.data() + 4 * (T.ebase[kl] + T.eoff[base + t]);
                const int ne = T.eoff[base + t + 1] - T.eoff[base + t];
                // the previous edge layer: the encoder's (radius r0, none for i = k) for l = 1
                const int Rep = l == 1 ? (i < k ? r0 : -1) : r0 + l - 2;
                const int eprev = l > 0 ? ecount(a, Rep) : 0;
                const int np1 = l > 0 ? ncount(a, r0 + l - 1) : 0;
                for (int p = 0; p < ne; ++p) {
                    const int q = T.eorder[(size_t)a * E + p];
                    if (l == 0) {
                        ec[4 * p] = g.dst[q]; ec[4 * p + 1] = g.src[q]; ec[4 * p + 2] = q; ec[4 * p + 3] = t;
                    } else {
                        const int pd = T.npos[(size_t)a * M + g.dst[q]], ps = T.npos[(size_t)a * M + g.src[q]];
                        ec[4 * p] = pd < np1 ? T.noff[pbase + t] + pd : -1;
                        ec[4 * p + 1] = ps < np1 ? T.noff[pbase + t] + ps : -1;
                        ec[4 * p + 2] = q;
                        ec[4 * p + 3] = p < eprev ? T.eoff[pbase + t] + p : -1;
                    }
                }
            }
        }
}

static void build_tangents(const gm_graph& g, int K, int N, Tangents& T) {
    const int M = g.M, E = g.E, nu = g.nu;
    T.Rmax = K * N;
    const int R1 = T.Rmax + 1;
    std::vector<std::vector<int>> out(M);
    for (int q = 0; q < E; ++q) out[g.src[q]].push_back(g.dst[q]);
    T.norder.assign((size_t)nu * M, 0);
    T.npos.assign((size_t)nu * M, 0);
    T.ncnt.assign((size_t)nu * R1, 0);
    T.eorder.assign((size_t)nu * std::max(E, 1), 0);
    T.epos.assign((size_t)nu * std::max(E, 1), 0);
    T.ecnt.assign((size_t)nu * R1, 0);
    const int INF = 1 << 30;
    std::vector<int> hop(M), ehop(std::max(E, 1)), idx;
    for (int a = 0; a < nu; ++a) {
        std::fill(hop.begin(), hop.end(), INF);
        std::vector<int> q{g.act_node[a]};
        hop[g.act_node[a]] = 0;
        for (size_t h = 0; h < q.size(); ++h)
            for (int w : out[q[h]])
                if (hop[w] == INF) {
                    hop[w] = hop[q[h]] + 1;
                    q.push_back(w);
                }
        idx.resize(M);
        for (int n = 0; n < M; ++n) idx[n] = n;
        std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) { return hop[x] < hop[y]; });
        for (int p = 0; p < M; ++p) {
            T.norder[(size_t)a * M + p] = idx[p];
            T.npos[(size_t)a * M + idx[p]] = p;
        }
        for (int n = 0; n < M; ++n)
            if (hop[n] <= T.Rmax) T.ncnt[(size_t)a * R1 + hop[n]]++;
        for (int R = 1; R < R1; ++R) T.ncnt[(size_t)a * R1 + R] += T.ncnt[(size_t)a * R1 + R - 1];
        if (E > 0) {
            for (int q2 = 0; q2 < E; ++q2) ehop[q2] = std::min(hop[g.src[q2]], hop[g.dst[q2]]);
            idx.resize(E);
            for (int q2 = 0; q2 < E; ++q2) idx[q2] = q2;
            std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) { return ehop[x] < ehop[y]; });
            for (int p = 0; p < E; ++p) {
                T.eorder[(size_t)a * E + p] = idx[p];
                T.epos[(size_t)a * E + idx[p]] = p;
            }
            for (int q2 = 0; q2 < E; ++q2)
                if (ehop[q2] <= T.Rmax) T.ecnt[(size_t)a * R1 + ehop[q2]]++;
            for (int R = 1; R < R1; ++R) T.ecnt[(size_t)a * R1 + R] += T.ecnt[(size_t)a * R1 + R - 1];
        }
    }
    const int L = N * nu + 1;
    T.noff.assign((size_t)N * (K + 1) * L, 0);
    T.eoff.assign((size_t)N * (K + 1) * L, 0);
    T.max_nrows = T.max_erows = 0;
    for (int k = 0; k < N; ++k)
        for (int l = 0; l <= K; ++l) {
            const size_t base = (size_t)(k * (K + 1) + l) * L;
            long on = 0, oe = 0;
            for (int t = 0; t < (k + 1) * nu; ++t) {
                const int i = t / nu, a = t % nu, r0 = K * (k - i);
                T.noff[base + t] = (int)on;
                T.eoff[base + t] = (int)oe;
                on += T.ncnt[(size_t)a * R1 + std::min(r0 + l, T.Rmax)];
                const int Re = l == 0 ? (i < k ? r0 : -1) : r0 + l - 1;
                if (Re >= 0 && E > 0) oe += T.ecnt[(size_t)a * R1 + std::min(Re, T.Rmax)];
            }
            T.noff[base + (k + 1) * nu] = (int)on;
            T.eoff[base + (k + 1) * nu] = (int)oe;
            T.max_nrows = std::max(T.max_nrows, on);
            T.max_erows = std::max(T.max_erows, oe);
        }
    build_tangent_ctx(g, K, N, T);
    T.aptr[T.aptr.size() - 1] = (int)T.alist.size();
}

static void build_cones(const gm_graph& g, int K, Cones& C) {
    const int M = g.M;
    C.K = K;
    C.nr_node.assign(K + 1, {});
    C.nr_seed.assign(K + 1, {});
    C.nr_ptr.assign(K + 1, {});
    C.nr_prev.assign(K + 1, {});
    C.er_edge.assign(K, {});
    C.er_dstrow.assign(K, {});
    C.er_srcrow.assign(K, {});
    C.er_prev.assign(K, {});
    C.er_dst_ptr.assign(K, {});
    C.er_src_ptr.assign(K, {});
    C.er_src_list.assign(K, {});
    std::vector<std::vector<std::pair<int, int>>> cone(M);
    std::vector<int> dist(M, -1), frontier, next, touched;
    for (int s = 0; s < M; ++s) {
        touched.assign(1, s);
        dist[s] = 0;
        frontier.assign(1, s);
        for (int d = 1; d <= K; ++d) {
            next.clear();
            for (int n : frontier)
                for (int e = g.in_ptr[n]; e < g.in_ptr[n + 1]; ++e) {
                    const int j = g.src[e];
                    if (dist[j] < 0) {
                        dist[j] = d;
                        touched.push_back(j);
                        next.push_back(j);
                    }
                }
            frontier.swap(next);
        }
        for (int n : touched) cone[s].push_back({n, dist[n]});
        std::sort(cone[s].begin(), cone[s].end());
        for (int n : touched) dist[n] = -1;
    }
    for (int r = 0; r <= K; ++r) {
        C.nr_ptr[r].push_back(0);
        for (int s = 0; s < M; ++s) {
            for (auto& nd : cone[s])
                if (nd.second <= r) {
                    C.nr_node[r].push_back(nd.first);
                    C.nr_seed[r].push_back(s);
                }
            C.nr_ptr[r].push_back((int)C.nr_node[r].size());
        }
        C.nr_prev[r].assign(C.nr_node[r].size(), -1);
        if (r > 0)
            for (size_t q = 0; q < C.nr_node[r].size(); ++q)
                C.nr_prev[r][q] = row_of(C.nr_node[r - 1], C.nr_ptr[r - 1], C.nr_seed[r][q], C.nr_node[r][q]);
    }
    for (int r = 0; r < K; ++r) {
        const int Rn = (int)C.nr_node[r].size();
        C.er_dst_ptr[r].assign(Rn + 1, 0);
        for (int q = 0; q < Rn; ++q) {
            C.er_dst_ptr[r][q] = (int)C.er_edge[r].size();
            const int s = C.nr_seed[r][q], i = C.nr_node[r][q];
            for (int e = g.in_ptr[i]; e < g.in_ptr[i + 1]; ++e) {
                C.er_edge[r].push_back(e);
                C.er_dstrow[r].push_back(q);
                C.er_srcrow[r].push_back(row_of(C.nr_node[r + 1], C.nr_ptr[r + 1], s, g.src[e]));
                int prev = -1;
                if (r > 0) {
                    const int qp = C.nr_prev[r][q];
                    if (qp >= 0) prev = C.er_dst_ptr[r - 1][qp] + (e - g.in_ptr[i]);
                }
                C.er_prev[r].push_back(prev);
            }
        }
        C.er_dst_ptr[r][Rn] = (int)C.er_edge[r].size();
        const int Rn1 = (int)C.nr_node[r + 1].size();
        std::vector<int> cnt(Rn1 + 1, 0);
        for (int sr : C.er_srcrow[r]) cnt[sr + 1]++;
        for (int q = 0; q < Rn1; ++q) cnt[q + 1] += cnt[q];
        C.er_src_ptr[r] = cnt;
        C.er_src_list[r].assign(C.er_edge[r].size(), 0);
        std::vector<int> fill(cnt.begin(), cnt.end() - 1);
        for (size_t p = 0; p < C.er_srcrow[r].size(); ++p) C.er_src_list[r][fill[C.er_srcrow[r][p]]++] = (int)p;
    }
    // encoder level: ER_{K-1} rows grouped by the NR_K row of their destination
    const int RK = (int)C.nr_node[K].size();
    std::vector<int> dK(C.er_edge[K - 1].size());
    for (size_t p = 0; p < dK.size(); ++p) {
        const int q = C.er_dstrow[K - 1][p];
        dK[p] = row_of(C.nr_node[K], C.nr_ptr[K], C.nr_seed[K - 1][q], C.nr_node[K - 1][q]);
    }
    C.enc_dst_ptr.assign(RK + 1, 0);
    for (int v : dK) C.enc_dst_ptr[v + 1]++;
    for (int q = 0; q < RK; ++q) C.enc_dst_ptr[q + 1] += C.enc_dst_ptr[q];
    C.enc_dst_list.assign(dK.size(), 0);
    {
        std::vector<int> fill(C.enc_dst_ptr.begin(), C.enc_dst_ptr.end() - 1);
        for (size_t p = 0; p < dK.size(); ++p) C.enc_dst_list[fill[dK[p]]++] = (int)p;
    }
    C.b_row.assign((size_t)M * g.nu, -1);
    for (int s = 0; s < M; ++s)
        for (int a = 0; a < g.nu; ++a) C.b_row[(size_t)s * g.nu + a] = row_of(C.nr_node[K], C.nr_ptr[K], s, g.act_node[a]);
}

// ---------------------------------------------------------------- weight layout
static long put(std::vector<float>& w, const float* p, size_t n) {
    while (w.size() % 32) w.push_back(0.f);
    long o = (long)w.size();
    w.insert(w.end(), p, p + n);
    return o;
}

// BF16 bit pattern of a float, round to nearest even (NaN kept quiet).
static uint16_t to_bf16(float f) {
    uint32_t u;
    std::memcpy(&u, &f, 4);
    if ((u & 0x7fffffffu) > 0x7f800000u) return 0x7fc0;
    u += 0x7fffu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}

// [rows][cols] matrix with entry (r, c) = f(r, c), appended 128-byte aligned.
static float from_bf16(uint16_t h) {
    uint32_t u = (uint32_t)h << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}

// The three BF16 pieces of a split tensor-core operand: p0 = bf16(f), p1 = bf16(f - p0),
// p2 = bf16(f - p0 - p1); p0 + p1 + p2 carries about 24 significant bits of f.  The
// [rows][cols] K-major operand with entry (r, c) = f(r, c) is stored in the tiled chunk
// layout (tc_tile_off) with chunk width kcw, 128-byte aligned; rows and cols are multiples of 16.
template <class F>
static long put_bf(std::vector<uint16_t>* wp, int rows, int cols, int kcw, F f) {
    while (wp[0].size() % 64)
        for (int p = 0; p < 3; ++p) wp[p].push_back(0);
    const long o = (long)wp[0].size();
    for (int p = 0; p < 3; ++p) wp[p].resize(o + (size_t)rows * cols, 0);
    for (int k0 = 0; k0 < cols; k0 += kcw) {
        const int kc = std::min(kcw, cols - k0);
        const long base = o + (long)rows * k0;
        for (int r = 0; r < rows; ++r)
            for (int c = 0; c < kc; ++c) {
                float v = f(r, k0 + c);
                for (int p = 0; p < 3; ++p) {
                    const uint16_t h = to_bf16(v);
                    wp[p][base + tc_tile_off(r, c, kc)] = h;
                    v -= from_bf16(h);
                }
            }
    }
    return o;
}

static void build_weights(const gm_gnn& m, int nu, std::vector<float>& w, std::vector<MlpOff>& offs,
                          std::vector<uint16_t>* wp) {
    const int K = m.d.K, W = m.d.W;
    std::vector<std::array<int, 3>> shapes;
    shapes.push_back({6 + nu, W, W});
    shapes.push_back({6, W, W});
    for (int t = 0; t < K; ++t) {
        shapes.push_back({3 * W, W, W});
        shapes.push_back({2 * W, W, W});
    }
    shapes.push_back({W, W, 3});
    const float* b = m.blob.data();
    size_t off = 0;
    offs.clear();
    for (size_t idx = 0; idx < shapes.size(); ++idx) {
        const int in = shapes[idx][0], hid = shapes[idx][1], out = shapes[idx][2];
        const float* W1 = b + off; off += (size_t)in * hid;
        const float* b1 = b + off; off += hid;
        const float* W2 = b + off; off += (size_t)hid * out;
        const float* b2 = b + off; off += out;
        MlpOff mo;
        mo.in = in; mo.hid = hid; mo.out = out;
        mo.W1 = put(w, W1, (size_t)in * hid);
        mo.b1 = put(w, b1, hid);
        mo.W2 = put(w, W2, (size_t)hid * out);
        mo.b2 = put(w, b2, out);
        std::vector<float> t((size_t)out * hid);
        for (int o = 0; o < out; ++o)
            for (int j = 0; j < hid; ++j) t[(size_t)o * hid + j] = W2[(size_t)j * out + o];
        mo.W2t = put(w, t.data(), t.size());
        t.assign((size_t)hid * in, 0.f);
        for (int j = 0; j < hid; ++j)
            for (int i = 0; i < in; ++i) t[(size_t)j * in + i] = W1[(size_t)i * hid + j];
        mo.W1t = put(w, t.data(), t.size());
        const bool edge_mp = idx >= 2 && idx < 2 + 2 * (size_t)K && (idx % 2 == 0);
        if (edge_mp) {
            t.assign((size_t)hid * W, 0.f);
            for (int j = 0; j < hid; ++j)
                for (int n = 0; n < W; ++n) t[(size_t)j * W + n] = W1[(size_t)(2 * W + n) * hid + j];
            mo.Wc = put(w, t.data(), t.size());
            t.assign((size_t)2 * W * W, 0.f);
            for (int j = 0; j < W; ++j)
                for (int n = 0; n < W; ++n) {
                    t[(size_t)j * W + n] = W1[(size_t)n * hid + j];
                    t[(size_t)(W + j) * W + n] = W1[(size_t)(W + n) * hid + j];
                }
            mo.Bab = put(w, t.data(), t.size());
            t.assign((size_t)W * 2 * W, 0.f);
            for (int k = 0; k < W; ++k)
                for (int n = 0; n < W; ++n) {
                    t[(size_t)k * 2 * W + n] = W1[(size_t)k * hid + n];
                    t[(size_t)k * 2 * W + W + n] = W1[(size_t)(W + k) * hid + n];
                }
            mo.Pab = put(w, t.data(), t.size());
            t.assign((size_t)W * W, 0.f);
            for (int k = 0; k < W; ++k) t[(size_t)k * W + k] = 1.f;
            mo.eye = put(w, t.data(), t.size());
        }
        // K-major BF16 operands of the tensor-core products (see MlpOff)
        auto up16 = [](int v) { return (v + 15) / 16 * 16; };
        mo.in_p = up16(in);
        mo.out_p = up16(out);
        mo.fk1 = put_bf(wp, hid, mo.in_p, TC_CHUNK_F, [&](int j, int i) { return i < in ? W1[(size_t)i * hid + j] : 0.f; });
        mo.fk2 = put_bf(wp, mo.out_p, hid, tc_chunk_b2_fwd(mo.out_p), [&](int o, int j) { return o < out ? W2[(size_t)j * out + o] : 0.f; });
        mo.bk1 = put_bf(wp, hid, mo.out_p, TC_CHUNK, [&](int j, int o) { return o < out ? W2[(size_t)j * out + o] : 0.f; });
        mo.bk2 = put_bf(wp, mo.in_p, hid, tc_chunk_b2(mo.in_p), [&](int i, int j) { return i < in ? W1[(size_t)i * hid + j] : 0.f; });
        if (edge_mp) {
            mo.wck = put_bf(wp, W, hid, tc_chunk_b2(W), [&](int n, int j) { return W1[(size_t)(2 * W + n) * hid + j]; });
            mo.babk = put_bf(wp, W, 2 * W, TC_CHUNK, [&](int n, int k) {
                return k < W ? W1[(size_t)n * hid + k] : W1[(size_t)(W + n) * hid + (k - W)];
            });
            mo.fck = put_bf(wp, hid, W, TC_CHUNK, [&](int j, int k) { return W1[(size_t)(2 * W + k) * hid + j]; });
            mo.pabk = put_bf(wp, 2 * W, W, tc_chunk_b2(2 * W), [&](int n, int k) {
                return n < W ? W1[(size_t)k * hid + n] : W1[(size_t)(W + k) * hid + (n - W)];
            });
            mo.eyek = put_bf(wp, W, W, TC_CHUNK, [&](int j, int k) { return j == k ? 1.f : 0.f; });
            mo.pabk1 = put_bf(wp, 2 * W, W, TC_CHUNK, [&](int n, int k) {
                return n < W ? W1[(size_t)k * hid + n] : W1[(size_t)(W + k) * hid + (n - W)];
            });
        }
        offs.push_back(mo);
    }
}

static size_t blob_floats(int K, int W, int nu) {
    auto mlp = [](size_t i, size_t h, size_t o) { return i * h + h + h * o + o; };
    size_t n = mlp(6 + nu, W, W) + mlp(6, W, W) + mlp(W, W, 3);
    n += (size_t)K * (mlp(3 * W, W, W) + mlp(2 * W, W, W));
    return n;
}

// ---------------------------------------------------------------- workspace layout
static constexpr int kMaxAdmmGrid = 2048;
static constexpr int kBatchLanes = 16;   // lanes of the pre parts of a batch step (gm_batch_rti_step)
static constexpr int kOverlapChunks = 4; // reverse-pass chunks of the horizon (overlap with the rollout)

static void plan(gm_ctx* c, Carver& cv) {
    const Cones& C = c->cones;
    const int M = c->M, E = c->E, K = c->K, W = c->W, N = c->N, nu = c->nu, nU = c->nU;
    const long RK = (long)C.nr_node[K].size(), RK1 = (long)C.nr_node[K - 1].size();
    const long RE = (long)C.er_edge[K - 1].size();
    // stages per reverse chunk: the per-chunk buffers within the budget (default 16 GB, which
    // holds the whole horizon of the chain of 1000 in one chunk: fewer, fuller launches measured
    // 7.9 ms for the Jacobian phase against 8.7 ms with 4-stage chunks)
    const long per_stage = 4L * (2 * RK * 3 * W + 2 * RK1 * 3 * W + 3 * RE * 3 * W + RK * 3 * (6 + nu) + RE * 18);
    const long budget = c->s.chunk_mb > 0 ? (long)c->s.chunk_mb << 20 : (16L << 30);
    c->stage_chunk = (int)std::max(1L, std::min((long)N, budget / std::max(1L, per_stage)));
    // by default chunks of at most a quarter of the horizon: the reverse pass of the first chunk
    // starts while the rollout of the later stages still runs (gnn_linearize)
    if (c->s.chunk_mb == 0) c->stage_chunk = std::min(c->stage_chunk, (N + kOverlapChunks - 1) / kOverlapChunks);
    // a matrix-free context steps without the reverse pass: gm_linearize still works on it, one
    // stage per launch group, with the smallest cotangent buffers
    if (c->s.condensing == 1 && c->s.chunk_mb == 0) c->stage_chunk = 1;
    const long Ns = c->stage_chunk;
    std::vector<float> wdummy;
    c->d_src = cv.take<int>(std::max(E, 1));
    c->d_dst = cv.take<int>(std::max(E, 1));
    c->d_in_ptr = cv.take<int>(M + 1);
    c->d_act = cv.take<int>(nu);
    c->d_jac_col = cv.take<int>(c->nnzb);
    c->d_wts = cv.take<float>(c->wts_host.size());
    for (int p = 0; p < 3; ++p) c->d_wbp[p] = cv.take<uint16_t>(std::max<size_t>(c->wbp_host[p].size(), 1));
    for (int r = 0; r <= K; ++r) {
        c->dc.nr_count[r] = (int)C.nr_node[r].size();
        c->dc.nr_node[r] = cv.take<int>(C.nr_node[r].size() + 1);
        c->dc.nr_prev[r] = cv.take<int>(C.nr_prev[r].size() + 1);
    }
    for (int r = 0; r < K; ++r) {
        c->dc.er_count[r] = (int)C.er_edge[r].size();
        c->dc.er_edge[r] = cv.take<int>(C.er_edge[r].size() + 1);
        c->dc.er_dstrow[r] = cv.take<int>(C.er_dstrow[r].size() + 1);
        c->dc.er_prev[r] = cv.take<int>(C.er_prev[r].size() + 1);
        c->dc.er_dst_ptr[r] = cv.take<int>(C.er_dst_ptr[r].size());
        c->dc.er_src_ptr[r] = cv.take<int>(C.er_src_ptr[r].size());
        c->dc.er_src_list[r] = cv.take<int>(C.er_src_list[r].size() + 1);
    }
    c->dc.enc_dst_ptr = cv.take<int>(C.enc_dst_ptr.size());
    c->dc.enc_dst_list = cv.take<int>(C.enc_dst_list.size() + 1);
    c->dc.nr_ptr_K = cv.take<int>(M + 1);
    c->dc.b_row = cv.take<int>((size_t)M * nu);
    const int ww = W / 32;
    c->d_h = cv.take<float>((size_t)M * W);
    c->d_e = cv.take<float>((size_t)std::max(E, 1) * W);
    c->d_agg = cv.take<float>((size_t)M * W);
    c->d_mask_node = cv.take<uint32_t>((size_t)N * (K + 2) * M * ww);
    c->d_mask_edge = cv.take<uint32_t>((size_t)N * (K + 1) * std::max(E, 1) * ww);
    c->d_dhA = cv.take<float>(Ns * RK * 3 * W);
    c->d_dhB = cv.take<float>(Ns * RK * 3 * W);
    c->d_dacc = cv.take<float>(Ns * RK1 * 3 * W);
    c->d_dagg = cv.take<float>(Ns * RK1 * 3 * W);
    c->d_deA = cv.take<float>(Ns * std::max(RE, 1L) * 3 * W);
    c->d_deB = cv.take<float>(Ns * std::max(RE, 1L) * 3 * W);
    c->d_ehid = cv.take<float>(Ns * std::max(RE, 1L) * 3 * W);
    c->d_dxn = cv.take<float>(Ns * RK * 3 * (6 + nu));
    c->d_dd = cv.take<float>(Ns * std::max(RE, 1L) * 18);
    c->d_u_hat = cv.take<float>((size_t)N * nu);
    c->d_x_hat = cv.take<float>((size_t)(N + 1) * M * 6);
    c->d_A = cv.take<float>((size_t)N * c->nnzb * 36);
    c->d_B = cv.take<float>((size_t)N * M * 6 * nu);
    c->d_c = cv.take<float>((size_t)N * M * 6);
    c->d_Cx = cv.take<float>(std::max(1L, c->rows_c * 3));
    c->d_dx = cv.take<float>(std::max(1L, c->rows_c));
    c->d_Gu = cv.take<float>((size_t)M * 6 * nu * ((size_t)N * (N + 1) / 2));
    c->d_Gx = cv.take<float>((size_t)(N + 1) * M * 6);
    c->d_defect = cv.take<float>((size_t)N * M * 6);
    c->d_H = cv.take<float>((size_t)nU * nU);
    c->d_g = cv.take<float>(nU);
    c->d_Ct = cv.take<float>(std::max(1L, c->ct_len));
    c->d_dt = cv.take<float>(std::max(1L, c->rows_c));
    c->d_U = cv.take<float>(nU);
    c->d_y = cv.take<float>(nU + c->rows_c);
    c->d_yw = cv.take<float>(nU + c->rows_c);
    c->d_z = cv.take<float>(nU + c->rows_c);
    c->d_rs = cv.take<float>(std::max(1L, c->rows_c));
    c->d_keep = cv.take<unsigned char>(std::max(1L, c->rows_c));
    c->d_kpos = cv.take<int>(std::max(1L, c->rows_c));
    c->d_kcnt = cv.take<int>(c->N);
    const long T = (nU + 31) / 32;
    c->d_gram_part = cv.take<float>(std::max((long)kGramSplitCap * T * T * 1024, 4L * 1024 * nU));
    c->d_L = cv.take<double>((size_t)factor_pad(nU) * factor_pad(nU));
    c->d_Linv = cv.take<double>((size_t)factor_pad(nU) * factor_pad(nU));
    c->d_P = cv.take<float>((size_t)nU * nU);
    c->d_Pinv = cv.take<float>((size_t)nU * nU);
    c->d_G = cv.take<float>((size_t)nU * nU);
    c->d_admm = cv.take<AdmmState>(1);
    c->d_acc = cv.take<float>(3 * (size_t)admm_acc_stride(nU));
    c->d_bar = cv.take<unsigned>(4);
    c->d_status = cv.take<int>(4);
    c->d_row_begin = cv.take<int>(kMaxAdmmGrid + 1);
    c->d_kkt = cv.take<double>(nU + 4);
    c->d_stats = cv.take<gm_stats>(1);
    c->d_ipm_rows = cv.take<double>((size_t)kIpmRowArrays * std::max(1L, c->rows_c));
    c->d_ipm_vec = cv.take<double>((size_t)kIpmVecArrays * nU + kIpmScalars);
    if (c->s.condensing == 1) {
        const Tangents& Tn = c->tan;
        c->dtan.norder = cv.take<int>(Tn.norder.size());
        c->dtan.npos = cv.take<int>(Tn.npos.size());
        c->dtan.ncnt = cv.take<int>(Tn.ncnt.size());
        c->dtan.eorder = cv.take<int>(Tn.eorder.size());
        c->dtan.epos = cv.take<int>(Tn.epos.size());
        c->dtan.ecnt = cv.take<int>(Tn.ecnt.size());
        c->dtan.noff = cv.take<int>(Tn.noff.size());
        c->dtan.eoff = cv.take<int>(Tn.eoff.size());
        c->dtan.nctx = cv.take<int4>(Tn.nctx.size() / 4 + 1);
        c->dtan.ectx = cv.take<int4>(Tn.ectx.size() / 4 + 1);
        c->dtan.aptr = cv.take<int>(Tn.aptr.size());
        c->dtan.alist = cv.take<int>(Tn.alist.size() + 1);
        c->d_thA = cv.take<float>((size_t)std::max(1L, Tn.max_nrows) * W);
        c->d_thB = cv.take<float>((size_t)std::max(1L, Tn.max_nrows) * W);
        c->d_tagg = cv.take<float>((size_t)std::max(1L, Tn.max_nrows) * W);
        c->d_teA = cv.take<float>((size_t)std::max(1L, Tn.max_erows) * W);
        c->d_teB = cv.take<float>((size_t)std::max(1L, Tn.max_erows) * W);
        c->d_tproj = cv.take<float>((size_t)std::max(1L, Tn.max_nrows) * 2 * W);
    }
}

}  // namespace gmi

using namespace gmi;

// ---------------------------------------------------------------- C ABI
extern "C" {

const char* gm_last_error(void) { return g_err.c_str(); }
const char* gm_version(void) { return "gnnmpc-b300 0.1 (sm_103a)"; }

gm_status gm_graph_create(int M, int E, const int32_t* src, const int32_t* dst, int nu,
                          const int32_t* act_node, gm_graph** out) {
    clear_error();
    GM_CHECK_ARG(out, "out is NULL");
    GM_CHECK_ARG(M >= 1, "M must be >= 1 (got %d)", M);
    GM_CHECK_ARG(E >= 0, "E must be >= 0 (got %d)", E);
    GM_CHECK_ARG(E == 0 || (src && dst), "src/dst are NULL");
    GM_CHECK_ARG(nu >= 1 && act_node, "nu must be >= 1 with act_node given");
    std::vector<std::pair<int, int>> ed(E);
    for (int k = 0; k < E; ++k) {
        GM_CHECK_ARG(src[k] >= 0 && src[k] < M && dst[k] >= 0 && dst[k] < M,
                     "edge %d (%d -> %d) out of range [0, %d)", k, src[k], dst[k], M);
        GM_CHECK_ARG(src[k] != dst[k], "edge %d is a self-loop", k);
        ed[k] = {dst[k], src[k]};
    }
    std::sort(ed.begin(), ed.end());
    for (int k = 1; k < E; ++k) GM_CHECK_ARG(ed[k] != ed[k - 1], "duplicate edge %d -> %d", ed[k].second, ed[k].first);
    for (int a = 0; a < nu; ++a) GM_CHECK_ARG(act_node[a] >= 0 && act_node[a] < M, "act_node[%d] = %d out of range", a, act_node[a]);
    auto* g = new gm_graph;
    g->M = M; g->E = E; g->nu = nu;
    g->src.resize(E); g->dst.resize(E);
    g->in_ptr.assign(M + 1, 0);
    for (int k = 0; k < E; ++k) {
        g->dst[k] = ed[k].first;
        g->src[k] = ed[k].second;
        g->in_ptr[ed[k].first + 1]++;
    }
    for (int i = 0; i < M; ++i) g->in_ptr[i + 1] += g->in_ptr[i];
    g->act_node.assign(act_node, act_node + nu);
    *out = g;
    return GM_OK;
}

void gm_graph_destroy(gm_graph* g) { delete g; }

gm_status gm_gnn_load(const gm_gnn_desc* d, const float* blob, size_t n, gm_gnn** out) {
    clear_error();
    GM_CHECK_ARG(d && blob && out, "NULL argument");
    GM_CHECK_ARG(d->K >= 1 && d->K <= 6, "K must be in [1, 6] (got %d)", d->K);
    GM_CHECK_ARG(d->W == 32 || d->W == 64 || d->W == 128, "W must be 32, 64 or 128 (got %d)", d->W);
    GM_CHECK_ARG(d->nu >= 1 && d->nu <= 64, "nu must be in [1, 64] (got %d)", d->nu);
    GM_CHECK_ARG(d->dt > 0.f, "dt must be > 0");
    const size_t need = blob_floats(d->K, d->W, d->nu);
    GM_CHECK_ARG(n == need, "blob has %zu floats, (K=%d, W=%d, nu=%d) needs %zu", n, d->K, d->W, d->nu, need);
    for (size_t i = 0; i < n; ++i) GM_CHECK_ARG(std::isfinite(blob[i]), "blob[%zu] is not finite", i);
    auto* m = new gm_gnn;
    m->d = *d;
    m->blob.assign(blob, blob + n);
    *out = m;
    return GM_OK;
}

void gm_gnn_destroy(gm_gnn* m) { delete m; }

static gm_status prepare(const gm_graph* g, const gm_gnn* m, const gm_settings* s, gm_ctx* c) {
    GM_CHECK_ARG(g && m && s, "NULL argument");
    GM_CHECK_ARG(g->nu == m->d.nu, "graph has nu=%d, GNN has nu=%d", g->nu, m->d.nu);
    GM_CHECK_ARG(s->N >= 1 && s->N <= 64, "N must be in [1, 64] (got %d)", s->N);
    GM_CHECK_ARG(s->n_c >= 0 && s->n_c <= 64, "n_c must be in [0, 64]");
    GM_CHECK_ARG(s->precision == GM_PREC_FP32 || s->precision == GM_PREC_MIXED || s->precision == GM_PREC_BF16,
                 "unknown precision %d", s->precision);
    GM_CHECK_ARG(s->rho > 0.f && s->tol > 0.f && s->max_iter >= 1, "rho, tol must be > 0 and max_iter >= 1");
    GM_CHECK_ARG(s->admm_grid >= 0 && s->factor_grid >= 0 && s->chunk_mb >= 0,
                 "admm_grid, factor_grid and chunk_mb must be >= 0");
    GM_CHECK_ARG((long)s->N * g->nu <= 256, "N * nu must be <= 256 (got %d)", s->N * g->nu);
    GM_CHECK_ARG(s->condensing == 0 || s->condensing == 1, "condensing must be 0 or 1 (got %d)", s->condensing);
    GM_CHECK_ARG(s->tan_split_rows >= 0, "tan_split_rows must be >= 0 (got %d)", s->tan_split_rows);
    c->s = *s;
    c->M = g->M; c->E = g->E; c->nu = g->nu; c->K = m->d.K; c->W = m->d.W; c->N = s->N;
    c->nU = s->N * g->nu; c->n_c = s->n_c; c->dt = m->d.dt;
    c->rows_c = (long)c->N * c->M * c->n_c;
    c->ct_len = (long)c->M * c->n_c * c->nu * ((long)c->N * (c->N + 1) / 2);
    c->graph = *g;
    build_cones(*g, c->K, c->cones);
    {   // the reverse node-sum keeps an edge range as first position | count << 24
        int maxc = 0;
        long maxp = 0;
        for (int r = 0; r < c->K; ++r) {
            const Cones& C = c->cones;
            for (size_t q = 0; q + 1 < C.er_dst_ptr[r].size(); ++q)
                maxc = std::max(maxc, C.er_dst_ptr[r][q + 1] - C.er_dst_ptr[r][q]);
            for (size_t q = 0; q + 1 < C.er_src_ptr[r].size(); ++q)
                maxc = std::max(maxc, C.er_src_ptr[r][q + 1] - C.er_src_ptr[r][q]);
            maxp = std::max(maxp, (long)C.er_edge[r].size());
        }
        GM_CHECK_ARG(maxc <= 255 && maxp < (1L << 24),
                     "graph too dense for the reverse pass: %d edges into or out of one node, %ld cone edges "
                     "(limits 255 and 2^24)", maxc, maxp);
    }
    c->jac_row_ptr = c->cones.nr_ptr[c->K];
    c->jac_col = c->cones.nr_node[c->K];
    c->nnzb = (int)c->jac_col.size();
    build_weights(*m, g->nu, c->wts_host, c->mlp, c->wbp_host);
    if (s->condensing == 1) {
        build_tangents(*g, c->K, c->N, c->tan);
        GM_CHECK_ARG(c->tan.max_nrows < (1L << 31) && c->tan.max_erows < (1L << 31),
                     "too many tangent rows for matrix-free condensing");
    }
    return GM_OK;
}

gm_status gm_ctx_workspace_size(const gm_graph* g, const gm_gnn* m, const gm_settings* s, size_t* bytes) {
    clear_error();
    GM_CHECK_ARG(bytes, "bytes is NULL");
    gm_ctx c;
    GM_TRY(prepare(g, m, s, &c));
    Carver cv;
    plan(&c, cv);
    *bytes = cv.off + 256;
    return GM_OK;
}

}  // extern "C"

template <class T>
static gm_status up(T* d, const std::vector<T>& h, cudaStream_t st) {
    if (h.empty()) return GM_OK;
    GM_CUDA_TRY(cudaMemcpyAsync(d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, st));
    return GM_OK;
}

extern "C" {

gm_status gm_ctx_create(const gm_graph* g, const gm_gnn* m, const gm_settings* s, void* workspace,
                        size_t bytes, void* stream, gm_ctx** out) {
    clear_error();
    GM_CHECK_ARG(out, "out is NULL");
    if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255)) {
        set_error("workspace is NULL or not 256-byte aligned");
        return GM_ERR_WORKSPACE;
    }
    auto* c = new gm_ctx;
    gm_status stt = prepare(g, m, s, c);
    if (stt != GM_OK) { delete c; return stt; }
    Carver probe;
    plan(c, probe);
    if (probe.off + 256 > bytes) {
        set_error("workspace has %zu bytes, needs %zu", bytes, probe.off + 256);
        delete c;
        return GM_ERR_WORKSPACE;
    }
    Carver cv;
    cv.base = static_cast<char*>(workspace);
    plan(c, cv);
    c->ws = static_cast<char*>(workspace);
    c->ws_bytes = bytes;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int dev = 0;
    auto fail = [&](gm_status e) { delete c; return e; };
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        set_error("no CUDA device: %s", cudaGetErrorString(cudaGetLastError()));
        return fail(GM_ERR_CUDA);
    }
    // the rollout's streams take the highest priority: its launches are short and dependent, and
    // the reverse pass that overlaps it would otherwise fill the SMs first
    int prio_lo = 0, prio_hi = 0;
    if (cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi) != cudaSuccess) {
        set_error("stream priority query failed: %s", cudaGetErrorString(cudaGetLastError()));
        return fail(GM_ERR_CUDA);
    }
    if (c->E > 0 && (cudaStreamCreateWithPriority(&c->side_stream, cudaStreamNonBlocking, prio_hi) != cudaSuccess ||
                     cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
                     cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess)) {
        set_error("side stream creation failed: %s", cudaGetErrorString(cudaGetLastError()));
        return fail(GM_ERR_CUDA);
    }
    const int n_chunks = (c->N + c->stage_chunk - 1) / c->stage_chunk;
    // matrix-free condensing: the tangent pass is the critical path and the rollout runs ahead of
    // it, so there the rollout takes the caller's priority and the tangent pass the highest
    // (closed-loop step 8.42 against 8.54 ms with the rollout at the highest priority)
    const int roll_prio = c->s.condensing == 1 ? prio_lo : prio_hi;
    if (c->s.condensing == 1 && (cudaStreamCreateWithPriority(&c->tan_stream, cudaStreamNonBlocking, prio_hi) != cudaSuccess ||
                                 cudaStreamCreateWithPriority(&c->tan_side, cudaStreamNonBlocking, prio_hi) != cudaSuccess ||
                                 cudaEventCreateWithFlags(&c->ev_tfork, cudaEventDisableTiming) != cudaSuccess ||
                                 cudaEventCreateWithFlags(&c->ev_tjoin, cudaEventDisableTiming) != cudaSuccess)) {
        set_error("tangent stream creation failed: %s", cudaGetErrorString(cudaGetLastError()));
        return fail(GM_ERR_CUDA);
    }
    if (cudaStreamCreateWithPriority(&c->roll_stream, cudaStreamNonBlocking, roll_prio) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_roll, cudaEventDisableTiming) != cudaSuccess) {
        set_error("rollout stream creation failed: %s", cudaGetErrorString(cudaGetLastError()));
        return fail(GM_ERR_CUDA);
    }
    for (int i = 0; i < n_chunks; ++i) {
        cudaEvent_t ev = nullptr;
        if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
            set_error("event creation failed: %s", cudaGetErrorString(cudaGetLastError()));
            return fail(GM_ERR_CUDA);
        }
        c->ev_stage.push_back(ev);
    }
    for (int i = 0; c->s.condensing == 1 && i < c->N; ++i) {
        cudaEvent_t ev = nullptr;
        if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
            set_error("event creation failed: %s", cudaGetErrorString(cudaGetLastError()));
            return fail(GM_ERR_CUDA);
        }
        c->ev_tan.push_back(ev);
    }
    if (c->s.condensing == 1 && cudaEventCreateWithFlags(&c->ev_tan_done, cudaEventDisableTiming) != cudaSuccess) {
        set_error("event creation failed: %s", cudaGetErrorString(cudaGetLastError()));
        return fail(GM_ERR_CUDA);
    }
    const Cones& C = c->cones;
    const int K = c->K;
    std::vector<gm_status> rs;
    rs.push_back(up(c->d_src, c->graph.src, st));
    rs.push_back(up(c->d_dst, c->graph.dst, st));
    rs.push_back(up(c->d_in_ptr, c->graph.in_ptr, st));
    rs.push_back(up(c->d_act, c->graph.act_node, st));
    rs.push_back(up(c->d_jac_col, c->jac_col, st));
    rs.push_back(up(c->d_wts, c->wts_host, st));
    for (int p = 0; p < 3; ++p) rs.push_back(up(c->d_wbp[p], c->wbp_host[p], st));
    for (int r = 0; r <= K; ++r) {
        rs.push_back(up(c->dc.nr_node[r], C.nr_node[r], st));
        rs.push_back(up(c->dc.nr_prev[r], C.nr_prev[r], st));
    }
    for (int r = 0; r < K; ++r) {
        rs.push_back(up(c->dc.er_edge[r], C.er_edge[r], st));
        rs.push_back(up(c->dc.er_dstrow[r], C.er_dstrow[r], st));
        rs.push_back(up(c->dc.er_prev[r], C.er_prev[r], st));
        rs.push_back(up(c->dc.er_dst_ptr[r], C.er_dst_ptr[r], st));
        rs.push_back(up(c->dc.er_src_ptr[r], C.er_src_ptr[r], st));
        rs.push_back(up(c->dc.er_src_list[r], C.er_src_list[r], st));
    }
    rs.push_back(up(c->dc.enc_dst_ptr, C.enc_dst_ptr, st));
    rs.push_back(up(c->dc.enc_dst_list, C.enc_dst_list, st));
    rs.push_back(up(c->dc.nr_ptr_K, C.nr_ptr[K], st));
    rs.push_back(up(c->dc.b_row, C.b_row, st));
    if (c->s.condensing == 1) {
        const Tangents& Tn = c->tan;
        rs.push_back(up(c->dtan.norder, Tn.norder, st));
        rs.push_back(up(c->dtan.npos, Tn.npos, st));
        rs.push_back(up(c->dtan.ncnt, Tn.ncnt, st));
        rs.push_back(up(c->dtan.eorder, Tn.eorder, st));
        rs.push_back(up(c->dtan.epos, Tn.epos, st));
        rs.push_back(up(c->dtan.ecnt, Tn.ecnt, st));
        rs.push_back(up(c->dtan.noff, Tn.noff, st));
        rs.push_back(up(c->dtan.eoff, Tn.eoff, st));
        rs.push_back(up(reinterpret_cast<int*>(c->dtan.nctx), Tn.nctx, st));
        rs.push_back(up(reinterpret_cast<int*>(c->dtan.ectx), Tn.ectx, st));
        rs.push_back(up(c->dtan.aptr, Tn.aptr, st));
        rs.push_back(up(c->dtan.alist, Tn.alist, st));
    }
    // ADMM: co-resident CTAs (cooperative launch); the row split is made on the device per solve
    {
        int occ = 0;
        if (cudaFuncSetAttribute(admm_kernel_ptr(c), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)admm_smem_bytes(c)) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, admm_kernel_ptr(c), ADMM_T, admm_smem_bytes(c)) !=
                cudaSuccess) {
            set_error("ADMM occupancy query failed: %s", cudaGetErrorString(cudaGetLastError()));
            return fail(GM_ERR_CUDA);
        }
        occ = std::max(occ, 1);
        long want = c->rows_c > 0 ? std::max(1L, std::min((long)occ * c->num_sms, c->rows_c / 16)) : 1;
        if (c->s.admm_grid > 0) want = std::min<long>(want, c->s.admm_grid);
        c->admm_grid = (int)std::min<long>(want, kMaxAdmmGrid);
        // every upload above reads host vectors that must outlive the copies
    }
    for (gm_status r : rs)
        if (r != GM_OK) return fail(r);
    if (cudaMemsetAsync(c->d_status, 0, sizeof(int) * 4, st) != cudaSuccess ||
        cudaMemsetAsync(c->d_u_hat, 0, sizeof(float) * c->N * c->nu, st) != cudaSuccess ||
        cudaMemsetAsync(c->d_y, 0, sizeof(float) * (c->nU + c->rows_c), st) != cudaSuccess ||
        cudaMemsetAsync(c->d_admm, 0, sizeof(AdmmState), st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        set_error("context upload failed: %s", cudaGetErrorString(cudaGetLastError()));
        return fail(GM_ERR_CUDA);
    }
    *out = c;
    return GM_OK;
}

void gm_ctx_destroy(gm_ctx* ctx) { delete ctx; }

gm_status gm_jac_pattern(const gm_ctx* ctx, int* nnzb, const int32_t** row_ptr, const int32_t** col) {
    clear_error();
    GM_CHECK_ARG(ctx && nnzb && row_ptr && col, "NULL argument");
    *nnzb = ctx->nnzb;
    *row_ptr = ctx->jac_row_ptr.data();
    *col = ctx->jac_col.data();
    return GM_OK;
}

gm_status gm_ctx_info(const gm_ctx* ctx, gm_info* o) {
    clear_error();
    GM_CHECK_ARG(ctx && o, "NULL argument");
    const gm_ctx* c = ctx;
    const Cones& C = c->cones;
    const double W = c->W, M = c->M, E = c->E, nu = c->nu, N = c->N, K = c->K;
    *o = gm_info{};
    o->M = c->M; o->E = c->E; o->nu = c->nu; o->K = c->K; o->W = c->W; o->N = c->N; o->n_c = c->n_c;
    o->nU = c->nU; o->nnzb = c->nnzb; o->rows_c = c->rows_c;
    for (int r = 0; r <= c->K; ++r) o->cone_node_rows += (long long)C.nr_node[r].size();
    for (int r = 0; r < c->K; ++r) o->cone_edge_rows += (long long)C.er_edge[r].size();
    // rollout: every MLP of every stage, 2 (in W + W out) flops per row
    double fwd = M * 2 * ((6 + nu) * W + W * W) + E * 2 * (6 * W + W * W) + M * 2 * (W * W + 3 * W);
    fwd += K * (E * 2 * (3 * W * W + W * W) + M * 2 * (2 * W * W + W * W));
    o->flops_rollout = N * fwd;
    // reverse pass over the cone rows (3 cotangent channels per row)
    double bwd = M * 3 * 2 * (3 * W + W * W);
    for (int r = 0; r < c->K; ++r) {
        const double nr = (double)C.nr_node[r].size(), er = (double)C.er_edge[r].size();
        const double nr1 = (double)C.nr_node[r + 1].size();
        bwd += nr * 3 * 2 * (W * W + W * 2 * W) + er * 3 * 2 * (W * W + W * W) + nr1 * 3 * 2 * (2 * W * W);
    }
    bwd += (double)C.nr_node[c->K].size() * 3 * 2 * (W * W + W * (6 + nu));
    bwd += (double)C.er_edge[c->K - 1].size() * 3 * 2 * (W * W + 6 * W);
    o->flops_jacobian = N * bwd;
    double cond = 0;
    for (int k = 1; k <= c->N; ++k) {
        const double L = k * nu;
        cond += c->nnzb * 36.0 * 2 * (L - nu + 1);          // recursion into stage k
        cond += M * 6 * L * (L + 1);                         // H (lower triangle), 2 flops each
        cond += M * 6 * 2 * L;                               // g
        cond += M * c->n_c * 2 * 3 * L;                      // C~ rows
    }
    o->flops_condense = cond;
    double setup = 0, iter = 0, bytes = 0;
    for (int k = 1; k <= c->N; ++k) {
        const double L = k * nu, rows = M * c->n_c;
        setup += rows * L * (L + 1);                         // C~'C~ lower triangle
        iter += rows * 2 * 2 * L;                            // C~ u and C~' w per row
        bytes += rows * (L * 4 + 4 + 8);                     // row, d~, z and y
    }
    const double n = c->nU;
    setup += n * n * n / 3 + n * n * n / 3 + n * n * n / 3;  // Cholesky, L^{-1}, L^{-T} L^{-1}
    iter += 2 * 2 * n * n;                                   // P^{-1} rhs and H U
    o->flops_qp_setup = setup;
    o->flops_admm_iter = iter;
    o->bytes_admm_iter = bytes;
    o->workspace_bytes = c->ws_bytes;
    o->stage_chunk = c->stage_chunk;
    o->admm_grid = c->admm_grid;
    return GM_OK;
}

gm_status gm_ctx_set_timing(gm_ctx* ctx, int on) {
    clear_error();
    GM_CHECK_ARG(ctx, "ctx is NULL");
    ctx->timing = on != 0;
    return GM_OK;
}

gm_status gm_ctx_phase_ms(gm_ctx* ctx, float* ms5, int* steps) {
    clear_error();
    GM_CHECK_ARG(ctx && ms5, "NULL argument");
    for (int p = 0; p < 5; ++p) ms5[p] = 0.f;
    for (auto& e : ctx->events) {
        GM_CUDA_TRY(cudaEventSynchronize(e[5]));
        for (int p = 0; p < 5; ++p) {
            float t = 0.f;
            GM_CUDA_TRY(cudaEventElapsedTime(&t, e[p], e[p + 1]));
            ms5[p] += t;
        }
    }
    if (steps) *steps = (int)ctx->events.size();
    for (auto& e : ctx->events)
        for (auto ev : e) cudaEventDestroy(ev);
    ctx->events.clear();
    return GM_OK;
}

unsigned long long gm_launch_count(void) { return g_launches.load(); }

gm_status gm_ctx_reset(gm_ctx* ctx, void* stream) {
    clear_error();
    GM_CHECK_ARG(ctx, "ctx is NULL");
    GM_CUDA_TRY(cudaMemsetAsync(ctx->d_u_hat, 0, sizeof(float) * ctx->N * ctx->nu, static_cast<cudaStream_t>(stream)));
    GM_CUDA_TRY(cudaMemsetAsync(ctx->d_y, 0, sizeof(float) * (ctx->nU + ctx->rows_c), static_cast<cudaStream_t>(stream)));
    GM_CUDA_TRY(cudaMemsetAsync(ctx->d_admm, 0, sizeof(AdmmState), static_cast<cudaStream_t>(stream)));
    return GM_OK;
}

gm_status gm_linearize(gm_ctx* ctx, const float* x0, const float* u_hat, float* x_hat, float* A, float* B,
                       float* c, void* stream) {
    clear_error();
    GM_CHECK_ARG(ctx && x0 && u_hat && x_hat, "NULL argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    GM_CUDA_TRY(cudaMemsetAsync(ctx->d_status + 2, 0, sizeof(int), st));
    GM_TRY(gnn_linearize(ctx, x0, u_hat, x_hat, A, B, c, st));
    return GM_OK;
}

gm_status gm_rollout(gm_ctx* ctx, const float* x0, const float* u, int n_steps, float* x_out, void* stream) {
    clear_error();
    GM_CHECK_ARG(ctx && x0 && u && x_out, "NULL argument");
    GM_CHECK_ARG(n_steps >= 1 && n_steps <= ctx->N, "n_steps must be in [1, N] (got %d)", n_steps);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    GM_CUDA_TRY(cudaMemsetAsync(ctx->d_status + 2, 0, sizeof(int), st));
    GM_TRY(gnn_rollout_steps(ctx, x0, u, x_out, n_steps, st));
    return GM_OK;
}

static gm_status check_cost(const gm_ctx* ctx, const gm_cost* cost, const gm_constr* cons) {
    GM_CHECK_ARG(cost && cost->Qdiag && cost->Rdiag && cost->x_ref && cost->u_ref, "cost has NULL members");
    GM_CHECK_ARG(cons && cons->u_lo && cons->u_hi, "constraints have NULL bounds");
    if (cons->n_spheres > 0) {
        GM_CHECK_ARG(cons->spheres, "spheres is NULL");
        GM_CHECK_ARG(cons->n_spheres == ctx->n_c, "n_spheres (%d) must equal settings.n_c (%d)", cons->n_spheres, ctx->n_c);
    } else if (ctx->n_c > 0) {
        GM_CHECK_ARG(cons->Cx && cons->dx, "Cx/dx are NULL with n_c = %d", ctx->n_c);
    }
    GM_CHECK_ARG(cons->barrier_mu >= 0.f && (cons->barrier_mu == 0.f || cons->barrier_delta > 0.f),
                 "barrier_mu must be >= 0, and barrier_delta > 0 when barrier_mu > 0 (got %g, %g)",
                 (double)cons->barrier_mu, (double)cons->barrier_delta);
    return GM_OK;
}

gm_status gm_condense(gm_ctx* ctx, const float* x_hat, const float* A, const float* B, const float* c,
                      const gm_cost* cost, const gm_constr* cons, float* H, float* g, float* Ct, float* dt,
                      void* stream) {
    clear_error();
    GM_CHECK_ARG(ctx && x_hat && A && B && c && H && g, "NULL argument");
    GM_TRY(check_cost(ctx, cost, cons));
    GM_CHECK_ARG(ctx->n_c == 0 || (Ct && dt), "Ct/dt are NULL with n_c = %d", ctx->n_c);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const float* Cx = cons->Cx;
    const float* dx = cons->dx;
    if (cons->n_spheres > 0) {
        GM_TRY(sphere_halfspaces(ctx, x_hat, cons->spheres, cons->n_spheres, ctx->d_Cx, ctx->d_dx, st));
        Cx = ctx->d_Cx;
        dx = ctx->d_dx;
    }
    return condense(ctx, x_hat, A, B, c, cost, Cx, dx, H, g, Ct, dt, st);
}

gm_status gm_condense_matrix_free(gm_ctx* ctx, const float* x0, const float* u_hat, const gm_cost* cost,
                                  const gm_constr* cons, float* x_hat, float* H, float* g, float* Ct, float* dt,
                                  void* stream) {
    clear_error();
    GM_CHECK_ARG(ctx && x0 && u_hat && x_hat && H && g, "NULL argument");
    GM_CHECK_ARG(ctx->s.condensing == 1, "the context was created with condensing = 0");
    GM_TRY(check_cost(ctx, cost, cons));
    GM_CHECK_ARG(ctx->n_c == 0 || (Ct && dt), "Ct/dt are NULL with n_c = %d", ctx->n_c);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    GM_TRY(gnn_rollout_sensitivities(ctx, x0, u_hat, x_hat, st));
    const float* Cx = cons->Cx;
    const float* dx = cons->dx;
    if (cons->n_spheres > 0) {
        GM_TRY(sphere_halfspaces(ctx, x_hat, cons->spheres, cons->n_spheres, ctx->d_Cx, ctx->d_dx, st));
        Cx = ctx->d_Cx;
        dx = ctx->d_dx;
    }
    return condense_tail(ctx, x_hat, cost, Cx, dx, H, g, Ct, dt, st);
}

gm_status gm_qp_solve(gm_ctx* ctx, const float* H, const float* g, const float* Ct, const float* dt,
                      const float* u_lo, const float* u_hi, const float* warm_U, const float* warm_y,
                      float* U, float* y, gm_stats* stats, void* stream) {
    clear_error();
    GM_CHECK_ARG(ctx && H && g && u_lo && u_hi && U, "NULL argument");
    GM_CHECK_ARG(!Ct == !dt, "Ct and dt must both be given or both be NULL (box only)");
    return qp_solve(ctx, H, g, Ct, dt, u_lo, u_hi, warm_U, warm_y, U, y, stats ? stats : ctx->d_stats,
                    static_cast<cudaStream_t>(stream));
}

// The two parts of one step: rti_pre (rollout, Jacobians, condensing, the warm start's duals)
// launches no cooperative kernel; rti_post (QP set-up, FP64 factorisation, ADMM, KKT check,
// outputs, the shift) holds the step's cooperative grids.  A batch runs the pre parts of many
// instances side by side and the post parts one after another (gm_batch_rti_step).
static gm_status rti_pre(gm_ctx* c, const float* x_meas, const gm_cost* cost, const gm_constr* cons, cudaStream_t st,
                         const std::array<cudaEvent_t, 6>* ev) {
    if (ev) GM_CUDA_TRY(cudaEventRecord((*ev)[0], st));
    GM_CUDA_TRY(cudaMemsetAsync(c->d_status + 2, 0, sizeof(int), st));
    c->kev_n = 0;
    const bool mf = c->s.condensing == 1;
    if (mf && ev) {   // matrix-free, phase timing: the rollout, then the sensitivities
        GM_TRY(gnn_rollout(c, x_meas, c->d_u_hat, c->d_x_hat, st));
        GM_CUDA_TRY(cudaEventRecord((*ev)[1], st));
        GM_TRY(gnn_sensitivities(c, c->d_u_hat, st));
        GM_CUDA_TRY(cudaEventRecord((*ev)[2], st));
    } else if (mf) {
        GM_TRY(gnn_rollout_sensitivities(c, x_meas, c->d_u_hat, c->d_x_hat, st));
    } else if (ev) {   // phase timing: the rollout and the reverse pass one after the other
        GM_TRY(gnn_rollout(c, x_meas, c->d_u_hat, c->d_x_hat, st));
        GM_CUDA_TRY(cudaEventRecord((*ev)[1], st));
        GM_TRY(gnn_jacobians(c, c->d_x_hat, c->d_u_hat, c->d_A, c->d_B, c->d_c, st));
        GM_CUDA_TRY(cudaEventRecord((*ev)[2], st));
    } else {
        GM_TRY(gnn_linearize(c, x_meas, c->d_u_hat, c->d_x_hat, c->d_A, c->d_B, c->d_c, st));
    }
    const float* Cx = cons->Cx;
    const float* dx = cons->dx;
    if (cons->n_spheres > 0) {
        GM_TRY(sphere_halfspaces(c, c->d_x_hat, cons->spheres, cons->n_spheres, c->d_Cx, c->d_dx, st));
        Cx = c->d_Cx;
        dx = c->d_dx;
    }
    if (mf) GM_TRY(condense_tail(c, c->d_x_hat, cost, Cx, dx, c->d_H, c->d_g, c->d_Ct, c->d_dt, st));
    else GM_TRY(condense(c, c->d_x_hat, c->d_A, c->d_B, c->d_c, cost, Cx, dx, c->d_H, c->d_g, c->d_Ct, c->d_dt, st));
    // barrier variant: the state rows go into the cost, the QP keeps the box
    const bool barrier = cons->barrier_mu > 0.f && c->n_c > 0;
    if (barrier)
        GM_TRY(barrier_fold(c, c->d_Ct, c->d_dt, c->d_u_hat, cons->barrier_mu, cons->barrier_delta, c->d_H, c->d_g,
                            st));
    // receding-horizon warm start: U^0 = u_hat (the shifted previous solution), y^0 = the previous
    // multipliers shifted by one stage alike (zero after gm_ctx_reset)
    if (c->warm) GM_TRY(shift_duals(c, c->d_y, c->d_yw, st));
    if (ev) GM_CUDA_TRY(cudaEventRecord((*ev)[3], st));
    return GM_OK;
}

static gm_status rti_post(gm_ctx* c, const gm_constr* cons, float* U, float* u0, gm_stats* stats, cudaStream_t st,
                          const std::array<cudaEvent_t, 6>* ev) {
    const bool barrier = cons->barrier_mu > 0.f && c->n_c > 0;
    GM_TRY(qp_solve(c, c->d_H, c->d_g, barrier ? nullptr : c->d_Ct, barrier ? nullptr : c->d_dt, cons->u_lo,
                    cons->u_hi, c->warm ? c->d_u_hat : nullptr, c->warm ? c->d_yw : nullptr, c->d_U, c->d_y,
                    stats ? stats : c->d_stats, st, ev ? (*ev)[4] : nullptr, c->warm));
    if (ev) GM_CUDA_TRY(cudaEventRecord((*ev)[5], st));
    GM_CUDA_TRY(cudaMemcpyAsync(U, c->d_U, sizeof(float) * c->nU, cudaMemcpyDeviceToDevice, st));
    if (u0) GM_CUDA_TRY(cudaMemcpyAsync(u0, c->d_U, sizeof(float) * c->nu, cudaMemcpyDeviceToDevice, st));
    GM_TRY(shift_inputs(c, c->d_U, c->d_u_hat, st));
    return GM_OK;
}

static gm_status rti_body(gm_ctx* c, const float* x_meas, const gm_cost* cost, const gm_constr* cons, float* U,
                          float* u0, gm_stats* stats, cudaStream_t st, bool timed) {
    std::array<cudaEvent_t, 6> ev{};
    if (timed) {
        for (auto& e : ev) GM_CUDA_TRY(cudaEventCreate(&e));
        c->events.push_back(ev);
    }
    GM_TRY(rti_pre(c, x_meas, cost, cons, st, timed ? &ev : nullptr));
    return rti_post(c, cons, U, u0, stats, st, timed ? &ev : nullptr);
}

// Everything a captured step bakes in.
static std::vector<uintptr_t> graph_key(const gm_ctx* c, const float* x_meas, const gm_cost* cost,
                                        const gm_constr* cons, float* U, float* u0, gm_stats* stats) {
    auto P = [](const void* p) { return reinterpret_cast<uintptr_t>(p); };
    std::vector<uintptr_t> k = {P(x_meas), P(cost->Qdiag), P(cost->Rdiag), P(cost->x_ref), P(cost->u_ref),
                                P(cons->u_lo), P(cons->u_hi), P(cons->Cx), P(cons->dx), (uintptr_t)cons->n_spheres,
                                P(cons->spheres), P(U), P(u0), P(stats)};
    uint32_t rho, tol, bmu, bdelta;
    std::memcpy(&rho, &c->s.rho, 4);
    std::memcpy(&tol, &c->s.tol, 4);
    std::memcpy(&bmu, &cons->barrier_mu, 4);
    std::memcpy(&bdelta, &cons->barrier_delta, 4);
    k.insert(k.end(), {(uintptr_t)bmu, (uintptr_t)bdelta, (uintptr_t)c->warm});
    k.insert(k.end(), {(uintptr_t)rho, (uintptr_t)tol, (uintptr_t)c->s.max_iter, (uintptr_t)c->s.scale_rows,
                       (uintptr_t)c->s.adapt_rho, (uintptr_t)c->s.timeout_spins, (uintptr_t)c->s.polish});
    return k;
}

// One step of c with these arguments captured into a graph on c's internal stream; part 0:
// the whole step, 1: rti_pre only, 2: rti_post only.
static gm_status capture_step(gm_ctx* c, const float* x_meas, const gm_cost* cost, const gm_constr* cons, float* U,
                              float* u0, gm_stats* stats, cudaGraph_t* out, int part = 0) {
    *out = nullptr;
    if (!c->cap_stream) GM_CUDA_TRY(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
    if (!c->cond_stream) GM_CUDA_TRY(cudaStreamCreateWithFlags(&c->cond_stream, cudaStreamNonBlocking));
    GM_CUDA_TRY(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeRelaxed));
    gm_status body = GM_OK;
    // the whole-step graph skips ADMM rounds after convergence through IF nodes; the batch's
    // per-lane pieces (parts 1 and 2) become child graphs and launch every round
    c->cond_capture = part == 0;
    if (part == 0) body = rti_body(c, x_meas, cost, cons, U, u0, stats, c->cap_stream, false);
    else if (part == 1) body = rti_pre(c, x_meas, cost, cons, c->cap_stream, nullptr);
    else body = rti_post(c, cons, U, u0, stats, c->cap_stream, nullptr);
    c->cond_capture = false;
    cudaGraph_t g = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(c->cap_stream, &g);
    if (body != GM_OK || ce != cudaSuccess || !g) {
        if (g) cudaGraphDestroy(g);
        (void)cudaGetLastError();
        if (body == GM_OK) set_error("stream capture failed: %s", cudaGetErrorString(ce));
        return body != GM_OK ? body : GM_ERR_CUDA;
    }
    *out = g;
    return GM_OK;
}

gm_status gm_rti_step(gm_ctx* ctx, const float* x_meas, const gm_cost* cost, const gm_constr* cons, float* U,
                      float* u0, gm_stats* stats, void* stream) {
    clear_error();
    GM_CHECK_ARG(ctx && x_meas && U, "NULL argument");
    GM_TRY(check_cost(ctx, cost, cons));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    gm_ctx* c = ctx;
    const bool timed = c->timing && c->events.size() < 100000;
    c->graph_replayed = false;
    if (!c->graph_on || c->graph_failed || timed) return rti_body(c, x_meas, cost, cons, U, u0, stats, st, timed);
    auto key = graph_key(c, x_meas, cost, cons, U, u0, stats);
    if (c->graph_exec && key == c->graph_key) {
        GM_CUDA_TRY(cudaGraphLaunch(c->graph_exec, st));
        c->graph_replayed = true;
        return GM_OK;
    }
    if (c->graph_eager++ == 0) return rti_body(c, x_meas, cost, cons, U, u0, stats, st, false);
    // capture on an internal stream (the caller's may be the legacy default stream), replay on st
    cudaGraph_t g = nullptr;
    cudaGraphExec_t exec = nullptr;
    if (capture_step(c, x_meas, cost, cons, U, u0, stats, &g) == GM_OK && cudaGraphInstantiate(&exec, g, cudaGraphInstantiateFlagUseNodePriority) == cudaSuccess) {
        cudaGraphDestroy(g);
        if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
        c->graph_exec = exec;
        c->graph_key = key;
        ++c->graph_captures;
        GM_CUDA_TRY(cudaGraphLaunch(c->graph_exec, st));
        c->graph_replayed = true;
        return GM_OK;
    }
    // capture unsupported here: eager steps from now on
    if (g) cudaGraphDestroy(g);
    (void)cudaGetLastError();
    c->graph_failed = true;
    return rti_body(c, x_meas, cost, cons, U, u0, stats, st, false);
}

gm_status gm_ws_features(gm_ctx* ctx, const float* x_meas, const float* x_ref, float* feat, void* stream) {
    clear_error();
    GM_CHECK_ARG(ctx && x_meas && x_ref && feat, "NULL argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    GM_TRY(gnn_latents(ctx, x_meas, ctx->d_u_hat, st));
    GM_TRY(ws_features(ctx, ctx->d_h, x_ref, feat, st));
    return GM_OK;
}

gm_status gm_batch_create(gm_ctx* const* ctxs, int n, gm_batch** out) {
    clear_error();
    GM_CHECK_ARG(ctxs && out && n >= 1, "NULL argument or empty batch");
    for (int i = 0; i < n; ++i) {
        GM_CHECK_ARG(ctxs[i], "ctxs[%d] is NULL", i);
        for (int j = 0; j < i; ++j) GM_CHECK_ARG(ctxs[j] != ctxs[i], "ctxs[%d] repeats ctxs[%d]", i, j);
    }
    gm_batch* b = new gm_batch;
    b->ctx.assign(ctxs, ctxs + n);
    // side by side, instances fill the GPU: programmatic early launches would only hold SMs
    for (int i = 0; i < n; ++i) {
        ctxs[i]->pdl = false;
        ctxs[i]->gram_tc = false;
        ctxs[i]->graph_key.clear();      // a context graph captured earlier is re-captured without it
    }
    *out = b;
    return GM_OK;
}

void gm_batch_destroy(gm_batch* b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    delete b;
}

gm_status gm_batch_rti_step(gm_batch* b, const float* const* x_meas, const gm_cost* costs, const gm_constr* cons,
                            float* const* U, gm_stats* const* stats, void* stream) {
    clear_error();
    GM_CHECK_ARG(b && x_meas && costs && cons && U, "NULL argument");
    const int n = (int)b->ctx.size();
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    std::vector<uintptr_t> key;
    for (int i = 0; i < n; ++i) {
        GM_CHECK_ARG(x_meas[i] && U[i], "instance %d: NULL argument", i);
        GM_TRY(check_cost(b->ctx[i], &costs[i], &cons[i]));
        auto k = graph_key(b->ctx[i], x_meas[i], &costs[i], &cons[i], U[i], nullptr, stats ? stats[i] : nullptr);
        key.insert(key.end(), k.begin(), k.end());
    }
    b->replayed = false;
    if (b->exec && key == b->key) {
        GM_CUDA_TRY(cudaGraphLaunch(b->exec, st));
        b->replayed = true;
        return GM_OK;
    }
    if (b->eager++ == 0) {        // first call: plain launches (one-time kernel attributes, cone uploads)
        for (int i = 0; i < n; ++i)
            GM_TRY(rti_body(b->ctx[i], x_meas[i], &costs[i], &cons[i], U[i], nullptr, stats ? stats[i] : nullptr,
                            st, false));
        return GM_OK;
    }
    // Every instance's step as two child graphs of one parent.  The pre parts (rollout,
    // Jacobians, condensing: no cooperative kernel) run in lanes side by side, planned by
    // gm_batch_plan on cost; the post parts (QP set-up, FP64 factorisation, ADMM, KKT: the
    // cooperative grids) follow their own pre part and run one after another in a single chain.
    // So at most one cooperative grid is on the GPU at a time: the non-cooperative kernels of
    // the other lanes always finish, so its CTAs all become resident and its grid barriers
    // wait for running CTAs only.  (Two cooperative grids side by side can each hold part of
    // their CTAs resident, every SM taken by spinning CTAs of one or the other, with the rest
    // of both waiting for an SM until a barrier's bound runs out.)
    std::vector<int> width(n, 1), lane(n);
    std::vector<double> cost(n);
    for (int i = 0; i < n; ++i) {
        const gm_ctx* c = b->ctx[i];
        cost[i] = (double)c->M * c->N * (1.0 + c->nU / 64.0);
    }
    int lanes = 1;
    GM_TRY(gm_batch_plan(n, width.data(), cost.data(), std::min(kBatchLanes, n), lane.data(), &lanes));
    if (b->lanes_req > 0 && b->lanes_req < lanes) {   // fewer lanes: instance i in lane i mod L
        lanes = b->lanes_req;
        for (int i = 0; i < n; ++i) lane[i] = i % lanes;
    }
    b->lanes = lanes;
    // post parts in the order their pre parts are expected to finish: by position in the lane,
    // the lanes round robin
    std::vector<int> pos(n, 0), seen(lanes, 0), order(n);
    for (int i = 0; i < n; ++i) pos[i] = seen[lane[i]]++;
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return pos[a] < pos[c]; });
    std::vector<int> tail(lanes, -1);
    cudaGraph_t parent = nullptr;
    GM_CUDA_TRY(cudaGraphCreate(&parent, 0));
    gm_status r = GM_OK;
    std::vector<cudaGraphNode_t> pre(n), post(n);
    auto add_child = [&](cudaGraphNode_t* node, const cudaGraphNode_t* deps, int nd, cudaGraph_t g, int i) {
        if (cudaGraphAddChildGraphNode(node, parent, deps, nd, g) != cudaSuccess) {
            set_error("adding instance %d to the batch graph failed", i);
            return GM_ERR_CUDA;
        }
        return GM_OK;
    };
    for (int i = 0; i < n && r == GM_OK; ++i) {
        cudaGraph_t g = nullptr;
        r = capture_step(b->ctx[i], x_meas[i], &costs[i], &cons[i], U[i], nullptr, stats ? stats[i] : nullptr, &g, 1);
        if (r != GM_OK) break;
        const cudaGraphNode_t* dep = tail[lane[i]] >= 0 ? &pre[tail[lane[i]]] : nullptr;
        tail[lane[i]] = i;
        r = add_child(&pre[i], dep, dep ? 1 : 0, g, i);
        cudaGraphDestroy(g);           // the child node holds its own copy
    }
    for (int j = 0; j < n && r == GM_OK; ++j) {
        const int i = order[j];
        cudaGraph_t g = nullptr;
        r = capture_step(b->ctx[i], x_meas[i], &costs[i], &cons[i], U[i], nullptr, stats ? stats[i] : nullptr, &g, 2);
        if (r != GM_OK) break;
        cudaGraphNode_t deps[2] = {pre[i], j > 0 ? post[order[j - 1]] : nullptr};
        r = add_child(&post[i], deps, j > 0 ? 2 : 1, g, i);
        cudaGraphDestroy(g);
    }
    cudaGraphExec_t exec = nullptr;
    if (r == GM_OK && cudaGraphInstantiate(&exec, parent, cudaGraphInstantiateFlagUseNodePriority) != cudaSuccess) {
        set_error("batch graph instantiation failed: %s", cudaGetErrorString(cudaGetLastError()));
        r = GM_ERR_CUDA;
    }
    cudaGraphDestroy(parent);
    if (r != GM_OK) return r;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = exec;
    b->key = std::move(key);
    ++b->captures;
    GM_CUDA_TRY(cudaGraphLaunch(b->exec, st));
    b->replayed = true;
    return GM_OK;
}

gm_status gm_batch_plan(int n, const int* width, const double* cost, int sms, int* lane, int* n_lanes) {
    clear_error();
    GM_CHECK_ARG(n >= 0 && sms >= 1, "n must be >= 0 and sms >= 1");
    GM_CHECK_ARG(n == 0 || (width && cost && lane && n_lanes), "NULL argument");
    if (!n_lanes) return GM_ERR_INVALID_ARG;
    *n_lanes = 0;
    for (int i = 0; i < n; ++i)
        GM_CHECK_ARG(width[i] >= 1 && cost[i] >= 0.0, "instance %d: width must be >= 1 and cost >= 0", i);
    if (n == 0) return GM_OK;
    // width classes, widest first; the narrowest class merges into the next wider one
    // until one lane per class fits (a single class wider than the SMs gets one lane)
    std::vector<int> cls;
    for (int i = 0; i < n; ++i) cls.push_back(std::min(width[i], sms));
    std::sort(cls.begin(), cls.end(), std::greater<int>());
    cls.erase(std::unique(cls.begin(), cls.end()), cls.end());
    auto sum = [&] { return std::accumulate(cls.begin(), cls.end(), 0L); };
    while (cls.size() > 1 && sum() > sms) cls.pop_back();
    const int nc = (int)cls.size();
    auto class_of = [&](int i) {     // the narrowest class at least as wide as the instance
        int k = 0;
        while (k + 1 < nc && cls[k + 1] >= std::min(width[i], sms)) ++k;
        return k;
    };
    std::vector<int> count(nc, 0), nl(nc, 1);
    std::vector<double> load(nc, 0.0);
    for (int i = 0; i < n; ++i) { ++count[class_of(i)]; load[class_of(i)] += cost[i]; }
    long left = sms - sum();
    for (;;) {                       // one more lane for the class with the largest load per lane
        int best = -1;
        for (int k = 0; k < nc; ++k)
            if (nl[k] < count[k] && cls[k] <= left && (best < 0 || load[k] * nl[best] > load[best] * nl[k]))
                best = k;
        if (best < 0) break;
        ++nl[best];
        left -= cls[best];
    }
    // longest processing time first inside each class: the costliest instance goes to the
    // least loaded of its class's lanes
    std::vector<int> first(nc, 0);
    for (int k = 1; k < nc; ++k) first[k] = first[k - 1] + nl[k - 1];
    std::vector<double> lane_load(first[nc - 1] + nl[nc - 1], 0.0);
    std::vector<int> order(n);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    for (int i : order) {
        const int k = class_of(i);
        int best = first[k];
        for (int l = first[k] + 1; l < first[k] + nl[k]; ++l)
            if (lane_load[l] < lane_load[best]) best = l;
        lane[i] = best;
        lane_load[best] += cost[i];
    }
    *n_lanes = (int)lane_load.size();
    return GM_OK;
}

gm_status gm_batch_set_lanes(gm_batch* b, int lanes) {
    clear_error();
    GM_CHECK_ARG(b && lanes >= 0, "NULL batch or lanes < 0");
    if (lanes != b->lanes_req) {
        b->lanes_req = lanes;
        b->key.clear();              // the next call captures the graph again
    }
    return GM_OK;
}

gm_status gm_batch_lanes(const gm_batch* b, int* lanes) {
    clear_error();
    GM_CHECK_ARG(b && lanes, "NULL argument");
    *lanes = b->lanes;
    return GM_OK;
}

gm_status gm_batch_state(const gm_batch* b, int* replayed, int* captures) {
    clear_error();
    GM_CHECK_ARG(b, "batch is NULL");
    if (replayed) *replayed = b->replayed ? 1 : 0;
    if (captures) *captures = b->captures;
    return GM_OK;
}

gm_status gm_ctx_set_warm(gm_ctx* ctx, int on) {
    clear_error();
    GM_CHECK_ARG(ctx, "ctx is NULL");
    ctx->warm = on != 0;
    return GM_OK;
}

gm_status gm_ctx_set_timeout_spins(gm_ctx* ctx, int spins) {
    clear_error();
    GM_CHECK_ARG(ctx, "ctx is NULL");
    GM_CHECK_ARG(spins >= 0, "spins must be >= 0 (got %d)", spins);
    ctx->s.timeout_spins = spins;       // part of a captured step's key: the next step re-captures
    return GM_OK;
}

gm_status gm_ctx_set_graph(gm_ctx* ctx, int on) {
    clear_error();
    GM_CHECK_ARG(ctx, "ctx is NULL");
    ctx->graph_on = on != 0;
    ctx->graph_failed = false;
    ctx->graph_eager = 0;
    if (!ctx->graph_on && ctx->graph_exec) {
        cudaGraphExecDestroy(ctx->graph_exec);
        ctx->graph_exec = nullptr;
        ctx->graph_key.clear();
    }
    return GM_OK;
}

gm_status gm_ctx_set_kernel_timing(gm_ctx* ctx, int on) {
    clear_error();
    GM_CHECK_ARG(ctx, "ctx is NULL");
    if ((on != 0) != ctx->ktiming && ctx->graph_exec) {     // the captured step changes: capture anew
        cudaGraphExecDestroy(ctx->graph_exec);
        ctx->graph_exec = nullptr;
        ctx->graph_key.clear();
    }
    ctx->ktiming = on != 0;
    ctx->kev_n = 0;
    return GM_OK;
}

gm_status gm_ctx_set_stage_timing(gm_ctx* ctx, int on) {
    clear_error();
    GM_CHECK_ARG(ctx, "ctx is NULL");
    GM_CHECK_ARG(ctx->s.condensing == 1, "stage timing needs a context created with gm_settings.condensing = 1");
    while (on && (int)ctx->sev.size() < 2 * ctx->N + 1) {
        cudaEvent_t ev;
        GM_CUDA_TRY(cudaEventCreate(&ev));
        ctx->sev.push_back(ev);
    }
    if ((on != 0) != ctx->stiming && ctx->graph_exec) {     // the captured step changes: capture anew
        cudaGraphExecDestroy(ctx->graph_exec);
        ctx->graph_exec = nullptr;
        ctx->graph_key.clear();
    }
    ctx->stiming = on != 0;
    return GM_OK;
}

gm_status gm_ctx_stage_times(gm_ctx* ctx, float* roll_ms, float* tan_ms) {
    clear_error();
    GM_CHECK_ARG(ctx && roll_ms && tan_ms, "NULL argument");
    GM_CHECK_ARG(ctx->stiming && (int)ctx->sev.size() >= 2 * ctx->N + 1, "stage timing is off");
    const int N = ctx->N;
    GM_CUDA_TRY(cudaEventSynchronize(ctx->sev[2 * N]));
    for (int k = 0; k < N; ++k) {
        GM_CUDA_TRY(cudaEventElapsedTime(&roll_ms[k], ctx->sev[0], ctx->sev[1 + k]));
        GM_CUDA_TRY(cudaEventElapsedTime(&tan_ms[k], ctx->sev[0], ctx->sev[1 + N + k]));
    }
    return GM_OK;
}

gm_status gm_ctx_kernel_stats(gm_ctx* ctx, int* launches, double* ms, double* bytes, double* flops) {
    clear_error();
    GM_CHECK_ARG(ctx && launches && ms && bytes && flops, "NULL argument");
    *launches = 0;
    *ms = *bytes = *flops = 0.0;
    for (int i = 0; i < ctx->kev_n && i < (int)ctx->kev.size(); ++i) {
        GM_CUDA_TRY(cudaEventSynchronize(ctx->kev[i][1]));
        float t = 0.f;
        GM_CUDA_TRY(cudaEventElapsedTime(&t, ctx->kev[i][0], ctx->kev[i][1]));
        *ms += t;
        *bytes += ctx->kev_bytes[i];
        *flops += ctx->kev_flops[i];
        ++*launches;
    }
    return GM_OK;
}

gm_status gm_ctx_kernel_launch(gm_ctx* ctx, int i, double* ms, double* bytes, int* ctas) {
    clear_error();
    GM_CHECK_ARG(ctx && ms && bytes && ctas, "NULL argument");
    GM_CHECK_ARG(i >= 0 && i < ctx->kev_n && i < (int)ctx->kev.size(), "launch index %d out of range", i);
    GM_CUDA_TRY(cudaEventSynchronize(ctx->kev[i][1]));
    float t = 0.f;
    GM_CUDA_TRY(cudaEventElapsedTime(&t, ctx->kev[i][0], ctx->kev[i][1]));
    *ms = t;
    *bytes = ctx->kev_bytes[i];
    *ctas = ctx->kev_ctas[i];
    return GM_OK;
}

gm_status gm_ctx_graph_state(const gm_ctx* ctx, int* replayed, int* captures) {
    clear_error();
    GM_CHECK_ARG(ctx, "ctx is NULL");
    if (replayed) *replayed = ctx->graph_replayed ? 1 : 0;
    if (captures) *captures = ctx->graph_captures;
    return GM_OK;
}

}  // extern "C"

namespace gmi {

// Algorithm 1 "update lin. trajectory": u_hat_k = U*_{k+1} (k < N-1), u_hat_{N-1} = U*_{N-1}.
// A solve that ended in NaN or gave up on a device wait leaves no usable U*: the trajectory
// then goes back to Algorithm 1's initial one (zeros), so that one failed step does not
// poison the steps after it.
__global__ void shift_kernel(int N, int nu, const float* __restrict__ U, float* __restrict__ u_hat,
                             const AdmmState* S) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N * nu) return;
    const int prev = S->final_status;
    if (prev == GM_ERR_NUMERIC || prev == GM_ERR_TIMEOUT) {
        u_hat[t] = 0.f;
        return;
    }
    int k = t / nu, a = t % nu;
    int src = k + 1 < N ? k + 1 : N - 1;
    u_hat[t] = U[src * nu + a];
}

gm_status shift_inputs(gm_ctx* c, const float* U, float* u_hat, cudaStream_t st) {
    shift_kernel<<<cdiv(c->N * c->nu, 128), 128, 0, st>>>(c->N, c->nu, U, u_hat, c->d_admm);
    GM_LAUNCH_CHECK();
    return GM_OK;
}

// The multipliers shifted like the inputs: box rows [N][nu] and half-space rows [N][M n_c]
// (stage-major) take stage k + 1's values, the last stage keeps its own.  After a solve that
// did not succeed (status other than GM_OK and GM_STALLED) the duals start at zero.
__global__ void shift_duals_kernel(int N, int nu, long Mnc, const float* __restrict__ y, float* __restrict__ yw,
                                   const AdmmState* S) {
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const long nU = (long)N * nu, total = nU + N * Mnc;
    if (t >= total) return;
    const int prev = S->final_status;
    if (prev != GM_OK && prev != GM_STALLED) {
        yw[t] = 0.f;
        return;
    }
    if (t < nU) {
        const int k = (int)(t / nu), a = (int)(t % nu);
        yw[t] = y[(long)(k + 1 < N ? k + 1 : N - 1) * nu + a];
    } else {
        const long r = t - nU;
        const int k = (int)(r / Mnc);
        yw[t] = y[nU + (long)(k + 1 < N ? k + 1 : N - 1) * Mnc + (r - (long)k * Mnc)];
    }
}

gm_status shift_duals(gm_ctx* c, const float* y, float* yw, cudaStream_t st) {
    const long Mnc = (long)c->M * c->n_c;
    const long total = c->nU + (long)c->N * Mnc;
    shift_duals_kernel<<<(unsigned)cdiv(total, 256L), 256, 0, st>>>(c->N, c->nu, Mnc, y, yw, c->d_admm);
    GM_LAUNCH_CHECK();
    return GM_OK;
}

}  // namespace gmi
