// Query planner and executor: the server side of the paper's Algorithm 2
// for the local threshold and InnerSum, with the attribute-selection product
// (Section 3.3), a private polynomial with encrypted coefficients, the
// encrypted threshold (Section 5.4.2), a composite odd sign polynomial mapped
// to step(x) = (sign(x) + 1)/2, the block sum and InnerSum (Appendix A.1.2
// rotations).
//
// Scale discipline: a ciphertext at level l carries S[l] (S[L] = Delta,
// S[l-1] = S[l]^2 / q_l), so a product of two level-l ciphertexts rescales
// exactly onto S[l-1].  adjust() moves a ciphertext to a lower level t with
// scale S[t] and applies a public factor a in one rescale: keep q_0..q_{t+1},
// multiply by floor(a * S[t] * q_{t+1} / scale + 1/2), rescale by q_{t+1}.
// Exceptions, kept exact by the planner: a power of x formed with a dropped
// (not adjusted) factor carries its factors' product over the removed prime;
// an encrypted coefficient multiplying a dropped power carries the ratio of
// scales from its arrival adjust; a sign stage folds its additive terms into
// the degree-2 sum before the relinearisation's rescale.  The circuit starts
// at the lowest level its depth allows and ends at level 1.
//
// A block group of nb blocks is evaluated with every launch covering all nb
// blocks (nb = all blocks: batched form; nb = 1: plain per-ciphertext form).
#include <algorithm>
#include <cstring>
#include <sstream>

#include "program.h"

namespace tetris {

// groups the w_j inputs are copied in (their transforms overlap the next group's copy)
constexpr int kInputChunks = 4;

struct QPlan {
    int l_lin, l_d, l_y, l_u, l_out;
    int l_ret = 1;  // the InnerSum and the returned ciphertext: drop to level 1 first
    bool ragged;
    double mask_scale;
    std::vector<std::vector<double>> co;
    double step_const;
    int degree = 0;
    int g = 0, m = 0, bb = 0, df = 0;  // baby-step giant-step schedule (g = 0: plain powers)
    // global threshold: folded stage coefficients (empty: none) and the record count R
    std::vector<std::vector<double>> gco;
    double records_norm = 0;
    // the circuit starts as low as its depth allows and ends at level 1: the
    // w_j are dropped from the top level to l_lin + 1, and the rescaled linear
    // combination has scale Delta pt_scale / q_{l_lin+1}, carried through the
    // powers of x by power_scales
    double x_scale = 0;
    // factor each c_k carries after its arrival adjust: the power it multiplies
    // is dropped (not rescaled) to the product's level lt, so c_k carries
    // S[lt] / S[level of the power] (and s_i's factor for x^(g i)); 1 where added
    std::vector<double> cfac;
    int coef_level(int k) const;
};

static int ceil_log2(int k) {
    int r = 0;
    while ((1 << r) < k) r++;
    return r;
}

// Baby-step giant-step form of y = sum_k c_k x^k with encrypted c_k:
//   y = s_0 + sum_{i>=1} s_i x^{g i},  s_i = sum_{j<g} c_{g i + j} x^j,
// g = 2^b, m = ceil((d+1)/g); every s_i (i >= 1) with a j >= 1 term is
// relinearised once, the degree-2 products of the last sum share one.
// Relinearisations: (g-2) + (m-1) + #{i >= 1 : g i + 1 <= d} + 1; the final
// products sit at depth D_f = max(ceil_log2(g-1) + 1, b + ceil_log2(m-1)).
// Taken when D_f <= ceil_log2(d) and it needs fewer than the d of plain
// powers (fewest relinearisations, then smallest g).
static void poly_schedule(QPlan &p, int d) {
    int best = -1;
    p.g = 0;
    for (int b = 1; b <= ceil_log2(d + 1); b++) {
        const int g = 1 << b, m = (d + 1 + g - 1) / g;
        if (m < 2) break;
        const int bb = ceil_log2(g - 1);
        const int df = std::max(bb + 1, b + ceil_log2(m - 1));
        if (df > ceil_log2(d)) continue;
        int relins = (g - 2) + (m - 1) + 1;
        for (int i = 1; i < m; i++) relins += (g * i + 1 <= d) ? 1 : 0;
        if (relins < d && (best < 0 || relins < best)) {
            best = relins;
            p.g = g; p.m = m; p.bb = bb; p.df = df;
        }
    }
}

// Scales and levels of y^1..y^n formed from y (scale, level) by the power rule
// y^k = y^a y^(k-a), a the largest power of two <= k (a power of two the square
// of its half), the lower factor dropped to the other's level and the
// relinearisation's rescale removing that level's prime.  Index k; [0] unused.
static void power_scales(const Ctx &C, double scale, int level, int n, std::vector<double> &sc, std::vector<int> &lv) {
    sc.assign(n + 1, 0.0);
    lv.assign(n + 1, 0);
    sc[1] = scale;
    lv[1] = level;
    for (int k = 2; k <= n; k++) {
        int a = 1;
        while (a * 2 <= k) a *= 2;
        const int A = a == k ? k / 2 : a, B = a == k ? k / 2 : k - a;
        sc[k] = (sc[A] * sc[B]) / (double)C.q[lv[A]];
        lv[k] = lv[A] - 1;
    }
}

// level at which the encrypted coefficient c_k is used
int QPlan::coef_level(int k) const {
    if (k == 0) return l_y;
    if (g == 0) return l_d;
    const int i = k / g, j = k % g;
    if (i == 0) return l_lin - df;          // s_0 terms, formed with the final products
    if (j >= 1) return l_lin - bb;          // tensors of s_i
    if (k + 1 <= degree) return l_lin - bb - 1;  // added to s_i after its relinearisation
    return l_lin - df;                      // s_i = c_k alone (k = d)
}

// levels a sign stage consumes: 3 for degree 7, 4 for degree 15
static int stage_depth(const std::vector<double> &co) {
    TREQUIRE(co.size() == 4 || co.size() == 8, TETRIS_EINVAL, "sign stages are odd polynomials of degree 7 or 15");
    return co.size() == 4 ? 3 : 4;
}

QPlan make_plan(const Ctx &C, uint64_t records, int degree, const std::vector<std::vector<double>> &stages,
                uint64_t norm_records = 0, const std::vector<std::vector<double>> &gstages = {}) {
    TREQUIRE(degree >= 1 && !stages.empty() && records >= 1, TETRIS_EINVAL, "empty query");
    QPlan p;
    const int L = C.L();
    const uint64_t n = C.N / 2;
    p.ragged = records % n != 0;
    // levels used below l_lin: polynomial, sign stages, ragged mask, global threshold
    int used = ceil_log2(degree) + 1 + (p.ragged ? 1 : 0);
    for (auto &co : stages) used += stage_depth(co);
    for (auto &co : gstages) used += stage_depth(co);
    p.l_lin = std::min(L - 1, 1 + used);
    p.l_d = p.l_lin - ceil_log2(degree);
    p.l_y = p.l_d - 1;
    p.l_u = p.l_y;
    for (auto &co : stages) p.l_u -= stage_depth(co);
    p.l_out = p.ragged ? p.l_u - 1 : p.l_u;
    TREQUIRE(p.l_out >= 1, TETRIS_ELEVEL, "circuit needs more levels: it would end at level " + std::to_string(p.l_out));
    const double R = (double)(norm_records ? norm_records : records);
    const size_t ns = stages.size();
    for (size_t s = 0; s < ns; s++) {
        std::vector<double> c = stages[s];
        if (s == 0)  // z = (y - t)/2 folded into the first stage
            for (size_t k = 0; k < c.size(); k++) c[k] = c[k] * std::ldexp(1.0, -(2 * (int)k + 1));
        if (s == ns - 1)  // step = (p + 1)/2, normalised by 1/records
            for (size_t k = 0; k < c.size(); k++) c[k] = c[k] / (2.0 * R);
        p.co.push_back(c);
    }
    p.step_const = 1.0 / (2.0 * R);
    p.x_scale = (C.S[L] * C.pt_scale) / (double)C.q[p.l_lin + 1];
    p.mask_scale = p.ragged ? (C.S[p.l_u - 1] * (double)C.q[p.l_u]) / C.S[p.l_u] : 0.0;
    p.degree = degree;
    poly_schedule(p, degree);
    {
        const auto &S = C.S;
        std::vector<double> sp, sg;
        std::vector<int> lp, lg;
        p.cfac.assign(degree + 1, 1.0);
        if (p.g == 0) {
            power_scales(C, p.x_scale, p.l_lin, degree, sp, lp);
        } else {
            power_scales(C, p.x_scale, p.l_lin, std::max(p.g - 1, 1), sp, lp);
            const int h = std::max(p.g / 2, 1);
            power_scales(C, (sp[h] * sp[h]) / (double)C.q[lp[h]], lp[h] - 1, std::max(p.m - 1, 1), sg, lg);
        }
        for (int k = 1; k <= degree; k++) {
            if (p.g == 0) {
                p.cfac[k] = S[p.l_d] / sp[k];
                continue;
            }
            const int i = k / p.g, j = k % p.g, l_b = p.l_lin - p.bb, l_f = p.l_lin - p.df;
            if (i == 0) {
                p.cfac[k] = S[l_f] / sp[j];
                continue;
            }
            // s_i multiplies x^(g i) dropped to l_f, and is itself dropped there
            // from l_b - 1 (its terms carry S[l_f] / S[l_b - 1] for that; c_d
            // alone, at l_f, does not)
            const double fi = S[l_f] / sg[i];
            const double rb = S[l_f] / S[l_b - 1];
            if (j >= 1) p.cfac[k] = (fi * (S[l_b] / sp[j])) * rb;
            else p.cfac[k] = k < degree ? fi * rb : fi;
        }
    }
    // global threshold: step = (p + 1)/2 folded into the last stage
    p.records_norm = R;
    for (size_t s = 0; s < gstages.size(); s++) {
        std::vector<double> c = gstages[s];
        if (s + 1 == gstages.size())
            for (size_t k = 0; k < c.size(); k++) c[k] = c[k] / 2.0;
        p.gco.push_back(c);
    }
    if (!p.gco.empty()) {
        p.l_ret = p.l_out;
        for (auto &co : p.gco) p.l_ret -= stage_depth(co);
        TREQUIRE(p.l_ret >= 1, TETRIS_ELEVEL,
                 "global threshold needs more levels: it would end at level " + std::to_string(p.l_ret));
    }
    return p;
}

static CtH relin_rescale_to(Rec &R, const CtH &t, int level_out) {
    CtH o = R.relin_rescale(t);
    o.scale = R.C.S[level_out];
    return o;
}

// The odd degree-7 part a0 u + [(a1 u) u^2 + ((a3 u) u^2 + a2 u) u^4] of a stage
// at level l, from the adjusts a = (a3 u at l-1, a2 u at l-2, a1 u at l-2,
// a0 u at l-3), u2 (l-1), u2d = u2 at l-2 and u4 (l-2): the two degree-2
// products in brackets formed at level l-2 and relinearised once; ends at l-3.
// T + a v for a degree-2 accumulator T at level lt (plaintext scale S[lt]^2)
// and a ciphertext v at level >= lt: v's first lt + 1 limbs times the integer
// round(a S[lt]^2 / scale(v)) added to T's first two components, no rescale
// (the relinearisation's rescale that follows covers it).  In place on T.
static CtH fold(Rec &R, const CtH &T, const CtH &v, double a) {
    Ctx &C = R.C;
    const int lt = T.level;
    TREQUIRE(T.comps == 3 && v.level >= lt && v.B == T.B, TETRIS_EINVAL, "fold: operands differ");
    const double cf = ((a * C.S[lt]) * C.S[lt]) / v.scale;
    TREQUIRE(std::fabs(cf) < 0x1p62, TETRIS_EINVAL, "fold: coefficient too large for an integer multiple");
    const int64_t c = round_half_up(cf);
    std::vector<EwJob> jobs;
    for (int i = 0; i <= lt; i++) {
        const u64 qi = C.q[i];
        EwJob proto{};
        proto.op = EW_ADD_MUL_CONST;
        proto.prime = i;
        proto.k = signed_mod(c, qi);
        proto.k_sh = h_shoup(proto.k, qi);
        for (int b = 0; b < T.B; b++)
            for (int k = 0; k < 2; k++) {
                EwJob j = proto;
                j.a = v.limb(b, k, i);
                j.b = j.dst = T.limb(b, k, i);
                jobs.push_back(j);
            }
    }
    R.ew(jobs);
    return T;
}

// One sign stage p(u) = sum_k a_k u^(2k+1): degree 7 in depth 3 as
// c0 u + [(a1 u) u^2 + ((a3 u) u^2 + c2 u) u^4] from the adjusts a3u (level
// l-1) and a1u (l-2), c2 u folded into (a3 u) u^2 before its
// relinearisation, c0 u into the bracket's two degree-2 products,
// relinearised once (ends at l-3): four relinearisations; degree 15 in
// depth 4 as A(u) + u^8 B(u), A and B the degree-7 parts of the low and
// high coefficients (u^2, u^4 shared), eight relinearisations, A folded into
// u^8 B.  The adjusts of u are independent: one pair of transforms; u^2 is
// only dropped.
static CtH sign_stage(Rec &R, const CtH &u, const std::vector<double> &co) {
    const int l = u.level;
    // u^2 is dropped to l-2 (scale S[l-1]); a1 u carries S[l-2] / S[l-1]
    const double r = R.C.S[l - 2] / R.C.S[l - 1];
    std::vector<Rec::AdjustItem> items = {{u, l - 1, co[3]}, {u, l - 2, co[1] * r}};
    if (co.size() == 8) {
        items.push_back({u, l - 1, co[7]});
        items.push_back({u, l - 2, co[5] * r});
    }
    std::vector<CtH> a = R.adjust_many(items);
    const bool deg15 = co.size() == 8;
    CtH u2 = R.mul(u, u);
    CtH u2d = R.drop(u2, l - 2);
    // the products of one depth are independent and share a level, so each
    // depth's relinearisations are one batched key switch (each ciphertext's
    // arithmetic as if relinearised alone): at level l-1 u^4 and the inner
    // products (a3 u) u^2 + a2 u of the degree-7 parts, at level l-2 their
    // outer sums (and u^8)
    std::vector<CtH> t1 = {R.tensor(u2, u2), fold(R, R.tensor(a[0], u2), u, co[2])};
    if (deg15) t1.push_back(fold(R, R.tensor(a[2], u2), u, co[6]));
    std::vector<CtH> r1 = R.relin_rescale_many(t1);
    for (CtH &x : r1) x.scale = R.C.S[l - 2];
    const CtH &u4 = r1[0];
    std::vector<CtH> t2 = {fold(R, R.tensor_add(R.tensor(a[1], u2d), r1[1], u4), u, co[0])};
    if (deg15) {
        t2.push_back(fold(R, R.tensor_add(R.tensor(a[3], u2d), r1[2], u4), u, co[4]));
        t2.push_back(R.tensor(u4, u4));
    }
    std::vector<CtH> r2 = R.relin_rescale_many(t2);
    for (CtH &x : r2) x.scale = R.C.S[l - 3];
    if (!deg15) return r2[0];
    return relin_rescale_to(R, fold(R, R.tensor(r2[2], r2[1]), r2[0], 1.0), l - 4);
}

// The circuit of nb blocks; stop (TETRIS_STAGE_*) ends it after a stage and
// returns that stage's ciphertexts.
static CtH eval_blocks(Rec &R, const Database &db, const QPlan &pl, int b0, int nb, const CtH &w,
                       const std::function<void()> &need_ck, const std::vector<CtH> &ck, const CtH &tadj, int degree,
                       int stop) {
    Ctx &C = R.C;
    const int tl = w.level;  // l_lin + 1
    const size_t N = C.N, nq = C.q.size();
    // x = sum_j pt_j * Enc(w_j), then rescale (the plaintexts' first tl + 1 limbs)
    CtH x0 = R.new_ct(nb, 2, tl);
    {
        // blocks innermost: the B jobs of one prime read the same w_j limbs back to back
        std::vector<LinJob> jobs;
        for (int i = 0; i <= tl; i++)
            for (int b = 0; b < nb; b++) {
                LinJob j{};
                j.pt = db.pts->ptr + (((size_t)(b0 + b) * db.attrs) * nq + i) * N;
                j.pt_stride = nq * N;
                j.w0 = w.limb(0, 0, i);
                j.w1 = w.limb(0, 1, i);
                j.w_stride = w.bstride;
                j.d0 = x0.limb(b, 0, i);
                j.d1 = x0.limb(b, 1, i);
                j.prime = i;
                j.nattr = db.attrs;
                jobs.push_back(j);
            }
        R.lin(jobs);
    }
    CtH x = R.rescale(x0);
    x.scale = pl.x_scale;
    x0 = CtH();
    if (stop == TETRIS_STAGE_X) return x;
    // powers x^k; a factor of lower power is dropped (not adjusted) to the
    // other's level, so a power's scale is its factors' product over the prime
    // the relinearisation removes (the planner's power_scales)
    std::map<int, CtH> Pw;
    Pw[1] = x;
    // x^k = x^a x^(k-a), a the largest power of two <= k (depth ceil_log2(k))
    auto power_rule = [&](std::map<int, CtH> &Q, int k) {
        int a = 1;
        while (a * 2 <= k) a *= 2;
        const CtH A = a == k ? Q[k / 2] : Q[a];
        const CtH B = a == k ? Q[k / 2] : R.drop(Q[k - a], A.level);
        CtH o = R.mul(A, B);
        o.scale = (A.scale * B.scale) / (double)C.q[A.level];
        return o;
    };
    CtH y;
    if (pl.g == 0) {
        for (int k = 2; k <= degree; k++) Pw[k] = power_rule(Pw, k);
        // y = sum_k c_k x^k with one relinearisation
        need_ck();
        CtH T;
        for (int k = 1; k <= degree; k++) T = R.tensor_add(T, ck[k], R.drop(Pw[k], pl.l_d));
        y = relin_rescale_to(R, T, pl.l_y);
    } else {
        const int g = pl.g, m = pl.m, l_b = pl.l_lin - pl.bb, l_f = pl.l_lin - pl.df;
        std::map<int, CtH> G;  // giant powers x^(g i)
        // the baby powers x^2 .. x^(g-1) and x^g = x^(g/2) x^(g/2), each by the power
        // rule; the products whose factors are ready and share a level are
        // relinearised by one batched key switch (the same arithmetic per power)
        {
            std::vector<int> todo;  // k < g: x^k; k == g: the first giant power
            for (int k = 2; k <= g; k++) todo.push_back(k);
            while (!todo.empty()) {
                std::map<int, std::vector<int>> by_level;  // ready powers by their factors' level
                std::map<int, std::pair<CtH, CtH>> fac;
                std::vector<int> rest;
                for (int k : todo) {
                    int a = 1;
                    while (a * 2 <= k) a *= 2;
                    const int ka = k == g ? g / 2 : (a == k ? k / 2 : a), kb = k == g ? g / 2 : (a == k ? k / 2 : k - a);
                    if (!Pw.count(ka) || !Pw.count(kb)) {
                        rest.push_back(k);
                        continue;
                    }
                    const CtH A = Pw[ka];
                    const CtH B = kb == ka ? A : R.drop(Pw[kb], A.level);
                    fac[k] = {A, B};
                    by_level[A.level].push_back(k);
                }
                TREQUIRE(!by_level.empty(), TETRIS_EINVAL, "power schedule: no power is ready");
                for (auto &lv : by_level) {
                    std::vector<CtH> ts;
                    for (int k : lv.second) ts.push_back(R.tensor(fac[k].first, fac[k].second));
                    std::vector<CtH> os = R.relin_rescale_many(ts);
                    for (size_t n = 0; n < lv.second.size(); n++) {
                        const int k = lv.second[n];
                        const CtH &A = fac[k].first, &B = fac[k].second;
                        os[n].scale = (A.scale * B.scale) / (double)C.q[A.level];
                        if (k == g) G[1] = os[n];
                        else Pw[k] = os[n];
                    }
                }
                todo = rest;
            }
        }
        for (int i = 2; i < m; i++) G[i] = power_rule(G, i);
        need_ck();
        CtH T;
        for (int j = 1; j < g; j++) T = R.tensor_add(T, ck[j], R.drop(Pw[j], l_f));  // s_0's terms at l_f
        // the inner sums s_i = c_(g i) + sum_j c_(g i + j) x^j, independent of one
        // another: their degree-2 sums relinearised by one batched key switch
        std::vector<CtH> Ts;
        std::vector<int> with_t;
        for (int i = 1; i < m; i++) {
            CtH Ti;
            for (int j = 1; j < g && g * i + j <= degree; j++) Ti = R.tensor_add(Ti, ck[g * i + j], R.drop(Pw[j], l_b));
            if (Ti.buf) {
                Ts.push_back(Ti);
                with_t.push_back(i);
            }
        }
        std::vector<CtH> rs = R.relin_rescale_many(Ts);
        for (int i = 1; i < m; i++) {
            CtH si = ck[g * i];
            const auto it = std::find(with_t.begin(), with_t.end(), i);
            if (it != with_t.end()) {
                CtH r = rs[it - with_t.begin()];
                r.scale = C.S[l_b - 1];
                si = R.drop(R.add(r, ck[g * i]), l_f);
            }
            T = R.tensor_add(T, si, R.drop(G[i], l_f));
        }
        G.clear();
        y = R.adjust(relin_rescale_to(R, T, l_f - 1), pl.l_y, 1.0);
    }
    Pw.clear();
    y = R.add(y, ck[0]);
    if (stop == TETRIS_STAGE_Y) return y;
    CtH u = R.sub(y, tadj);
    if (stop == TETRIS_STAGE_D) return u;
    for (auto &co : pl.co) u = sign_stage(R, u, co);
    return R.add_int(u, round_half_up(pl.step_const * C.S[u.level]));
}

// Limbs of an input at level `from` that an adjust to level lt reads: the
// first lt + 2 (keep q_0..q_{lt+1}, rescale by q_{lt+1}), or lt + 1 when it
// arrives at lt.  Dropping the others before the copy is exact.
static int used_limbs(int from, int lt) {
    TREQUIRE(from >= lt, TETRIS_ELEVEL, "input ciphertext level too low");
    return from == lt ? lt + 1 : lt + 2;
}

std::vector<InSlot> query_slot_shapes(const Ctx &C, const Database &db, const QuerySpec &q) {
    const QPlan pl = make_plan(C, db.records, q.degree, q.stages, q.total_records, q.gstages);
    const size_t N = C.N;
    std::vector<InSlot> v;
    auto add = [&](int from, int m) {
        InSlot s;
        s.rows = 2;
        s.row_words = (size_t)m * N;
        s.src_pitch = (size_t)(from + 1) * N;
        v.push_back(s);
    };
    for (int j = 0; j < q.attrs; j++) add(C.L(), pl.l_lin + 2);  // the w_j, dropped to l_lin + 1
    for (int k = 0; k <= q.degree; k++) add(q.c_level[k], used_limbs(q.c_level[k], pl.coef_level(k)));
    add(q.t_level, used_limbs(q.t_level, pl.l_y));
    if (!q.gstages.empty()) add(q.g_level, used_limbs(q.g_level, pl.l_out));
    return v;
}

std::unique_ptr<Program> record_query(Ctx &C, const Database &db, const QuerySpec &q) {
    auto P = std::make_unique<Program>();
    P->ctx = &C;
    Rec R(C, *P);
    R.persistent = q.persistent != 0;
    const QPlan pl = make_plan(C, db.records, q.degree, q.stages, q.total_records, q.gstages);
    const size_t N = C.N;
    // staging buffers for the inputs (coefficient domain on arrival, NTT in
    // place), holding only the limbs the circuit reads of each input
    P->in_slots = query_slot_shapes(C, db, q);
    const int lw = pl.l_lin + 1;  // the w_j's level after the drop
    const size_t wwords = P->in_slots[0].words();
    BufPtr wbuf = P->pool.alloc(wwords * q.attrs);
    P->hold.push_back(wbuf);
    for (int j = 0; j < q.attrs; j++) P->in_slots[j].dst = wbuf->ptr + j * wwords;
    size_t slot = q.attrs;
    auto input = [&](double scale) {
        InSlot &sl = P->in_slots[slot++];
        CtH c = R.new_ct(1, 2, (int)(sl.row_words / N) - 1);
        c.scale = scale;
        P->hold.push_back(c.buf);
        sl.dst = c.base;
        return c;
    };
    std::vector<CtH> cin;
    for (int k = 0; k <= q.degree; k++) cin.push_back(input(q.c_scale[k]));
    CtH tin = input(q.t_scale);
    CtH t1in;
    if (!q.gstages.empty()) t1in = input(q.g_scale);
    // per-query: the w_j (one batch of attrs ciphertexts) dropped to level
    // l_lin + 1, their remaining limbs to the NTT domain
    auto ntt_inputs = [&](const std::vector<CtH> &cts) {
        std::vector<NttJob> jobs;
        for (const CtH &c : cts)
            for (int b = 0; b < c.B; b++)
                for (int k = 0; k < c.comps; k++)
                    for (int i = 0; i <= c.level; i++) {
                        NttJob j{};
                        j.src = j.dst = c.limb(b, k, i);
                        j.prime = i;
                        jobs.push_back(j);
                    }
        R.ntt(false, jobs, LOAD_PLAIN, STORE_PLAIN);
    };
    CtH w = R.view(wbuf, wbuf->ptr, q.attrs, 2, lw, wwords, (size_t)(lw + 1) * N, C.S[C.L()]);
    // the w_j arrive in up to kInputChunks groups: each group's transforms wait
    // only for its own copy, so they overlap the next group's
    const int chunks = std::min(q.attrs, kInputChunks), per = (q.attrs + chunks - 1) / chunks;
    for (int j0 = 0; j0 < q.attrs; j0 += per) {
        const int j1 = std::min(q.attrs, j0 + per);
        if (j0 > 0) P->add_input_wait((size_t)j0);
        ntt_inputs({R.view(wbuf, wbuf->ptr + (size_t)j0 * wwords, j1 - j0, 2, lw, wwords, (size_t)(lw + 1) * N,
                           C.S[C.L()])});
    }
    // the coefficients and the threshold (and t1) are late inputs: their copies
    // overlap the linear combination and the first powers of x, and they are
    // brought to their levels and transformed where first used
    std::vector<CtH> ck;
    CtH tadj;
    auto need_ck = [&]() {
        if (!ck.empty()) return;
        P->add_input_wait((size_t)q.attrs);
        std::vector<Rec::AdjustItem> items;
        for (int k = 0; k <= q.degree; k++) items.push_back({cin[k], pl.coef_level(k), pl.cfac[k]});
        items.push_back({tin, pl.l_y, 1.0});
        ck = R.adjust_many_coef(items);
        tadj = ck.back();
        ck.pop_back();
        std::vector<CtH> all = ck;
        all.push_back(tadj);
        ntt_inputs(all);
    };
    // block groups
    const int B = db.blocks;
    const int bpl = q.bpl <= 0 ? B : std::min(q.bpl, B);
    CtH full, last;
    bool have_full = false, have_last = false;
    if (q.stage != TETRIS_STAGE_FULL) {
        // the stage's ciphertexts of every block, block after block, coefficient domain
        BufPtr ob;
        size_t bw = 0;
        for (int b0 = 0; b0 < B; b0 += bpl) {
            const int nb = std::min(bpl, B - b0);
            CtH v = eval_blocks(R, db, pl, b0, nb, w, need_ck, ck, tadj, q.degree, q.stage);
            if (!ob) {
                bw = (size_t)2 * (v.level + 1) * N;
                ob = P->pool.alloc(bw * B);
                P->out_level = v.level;
                P->out_scale = v.scale;
            }
            std::vector<NttJob> jobs;
            for (int b = 0; b < nb; b++)
                for (int c = 0; c < 2; c++)
                    for (int i = 0; i <= v.level; i++) {
                        NttJob j{};
                        j.src = v.limb(b, c, i);
                        j.dst = ob->ptr + (size_t)(b0 + b) * bw + ((size_t)c * (v.level + 1) + i) * N;
                        j.prime = i;
                        jobs.push_back(j);
                    }
            R.ntt(true, jobs, LOAD_PLAIN, STORE_PLAIN);
        }
        P->out_buf = ob;
        P->out_base = ob->ptr;
        P->out_words = bw * B;
        P->out_comps = 2;
        P->finalize();
        return P;
    }
    for (int b0 = 0; b0 < B; b0 += bpl) {
        const int nb = std::min(bpl, B - b0);
        CtH u = eval_blocks(R, db, pl, b0, nb, w, need_ck, ck, tadj, q.degree, TETRIS_STAGE_FULL);
        int nfull = nb;
        if (pl.ragged && b0 + nb == B) {
            last = R.view(u.buf, u.limb(nb - 1, 0, 0), 1, u.comps, u.level, u.bstride, u.cstride, u.scale);
            have_last = true;
            nfull = nb - 1;
        }
        if (nfull > 0) {
            CtH part = R.sum_batch(R.view(u.buf, u.base, nfull, u.comps, u.level, u.bstride, u.cstride, u.scale));
            full = have_full ? R.add(full, part) : part;
            have_full = true;
        }
    }
    CtH acc;
    if (pl.ragged) {
        TREQUIRE(db.mask_real && have_last, TETRIS_EINVAL, "database has no mask for its ragged last block");
        BufPtr mi = P->pool.alloc(N);
        BufPtr mpt = P->pool.alloc((size_t)(pl.l_u + 1) * N);
        const double *mr = reinterpret_cast<const double *>(db.mask_real->ptr);
        int64_t *mip = reinterpret_cast<int64_t *>(mi->ptr);
        const double ms = pl.mask_scale;
        P->add_launch([=](cudaStream_t s, const uint8_t *) { round_scale(mr, mip, N, ms, s); }, "round_scale", 16.0 * N);
        std::vector<NttJob> jobs;
        for (int i = 0; i <= pl.l_u; i++) {
            NttJob j{};
            j.src = mi->ptr;
            j.dst = mpt->ptr + (size_t)i * N;
            j.prime = i;
            jobs.push_back(j);
        }
        R.ntt(false, jobs, LOAD_INT64, STORE_PLAIN);
        CtH m = R.rescale(R.mul_plain(last, mpt->ptr, 0));
        m.scale = C.S[pl.l_out];
        acc = have_full ? R.add(R.adjust(full, pl.l_out, 1.0), m) : m;
    } else {
        acc = full;
    }
    // InnerSum: acc += Rot_{2^k}(acc), after dropping to level l_ret (the
    // rotations' key switches then work on two primes; the value, below
    // S[l_out] in magnitude, is far inside q_0 q_1) -- unless a global
    // threshold follows, which needs the levels
    double acc_scale = acc.scale;
    if (pl.gco.empty()) acc = R.drop(acc, std::min(acc.level, pl.l_ret));
    for (int k = 0; k + 1 < C.log_n; k++) {
        const uint32_t g = (uint32_t)h_powmod(5, 1ull << k, 2 * C.N);
        acc = R.add(acc, R.rotate(acc, g));
    }
    if (!pl.gco.empty()) {
        // global threshold (Algorithm 2, last line): step((count - t1 + 1/2) / R)
        // from acc = count / R; t1 enters as a count scaled by 1/R in its adjust
        const double R0 = pl.records_norm;
        CtH t1 = R.adjust_many_coef({{t1in, acc.level, 1.0 / R0}})[0];
        {
            std::vector<NttJob> jobs;
            for (int c = 0; c < 2; c++)
                for (int i = 0; i <= t1.level; i++) {
                    NttJob j{};
                    j.src = j.dst = t1.limb(0, c, i);
                    j.prime = i;
                    jobs.push_back(j);
                }
            R.ntt(false, jobs, LOAD_PLAIN, STORE_PLAIN);
        }
        CtH z = R.add_int(R.sub(acc, t1), round_half_up(C.S[acc.level] / (2.0 * R0)));
        for (auto &co : pl.gco) z = sign_stage(R, z, co);
        acc = R.add_int(z, round_half_up(0.5 * C.S[z.level]));
        acc_scale = C.S[acc.level];
    }
    CtH o = R.from_ntt(acc);
    P->out_buf = o.buf;
    P->out_base = o.base;
    P->out_words = o.bstride;
    P->out_level = acc.level;
    P->out_comps = 2;
    P->out_scale = acc_scale;
    P->finalize();
    return P;
}

QuerySpec spec_of(const Ctx &C, const Database &db, const tetris_query *q) {
    TREQUIRE(q && q->w && q->f_coeffs && q->threshold && q->sign_coeffs, TETRIS_EINVAL, "query: null pointer");
    TREQUIRE((int)q->n_attrs == db.attrs, TETRIS_EINVAL, "query: attribute count differs from the database");
    TREQUIRE(q->sign_degree == 7 || q->sign_degree == 15, TETRIS_EINVAL,
             "query: sign stages must be odd polynomials of degree 7 or 15");
    const uint32_t nco = (q->sign_degree + 1) / 2;
    TREQUIRE(q->sign_stages >= 1 && q->f_degree >= 1, TETRIS_EINVAL, "query: empty polynomial");
    QuerySpec s;
    s.attrs = q->n_attrs;
    s.degree = q->f_degree;
    const int L = C.L();
    for (uint32_t j = 0; j < q->n_attrs; j++) {
        TREQUIRE(q->w[j].level == (uint32_t)L && q->w[j].ncomp == 2 && q->w[j].scale == C.S[L] && q->w[j].data,
                 TETRIS_EINVAL, "query: linear-combination coefficients must be fresh top-level ciphertexts");
    }
    for (uint32_t k = 0; k <= q->f_degree; k++) {
        TREQUIRE(q->f_coeffs[k].ncomp == 2 && (int)q->f_coeffs[k].level <= L && q->f_coeffs[k].data && q->f_coeffs[k].scale > 0,
                 TETRIS_EINVAL, "query: bad polynomial coefficient ciphertext");
        s.c_level.push_back(q->f_coeffs[k].level);
        s.c_scale.push_back(q->f_coeffs[k].scale);
    }
    TREQUIRE(q->threshold->ncomp == 2 && (int)q->threshold->level <= L && q->threshold->data && q->threshold->scale > 0,
             TETRIS_EINVAL, "query: bad threshold ciphertext");
    s.t_level = q->threshold->level;
    s.t_scale = q->threshold->scale;
    for (uint32_t st = 0; st < q->sign_stages; st++)
        s.stages.push_back(std::vector<double>(q->sign_coeffs + st * nco, q->sign_coeffs + (st + 1) * nco));
    s.bpl = C.blocks_per_launch;
    s.loge = C.nt.loge;
    s.stage = C.query_stage;
    s.persistent = C.persistent;
    TREQUIRE(q->total_records == 0 || q->total_records >= db.records, TETRIS_EINVAL,
             "query: total_records is smaller than the database");
    s.total_records = q->total_records;
    if (q->global_threshold) {
        const tetris_ct_in &g = *q->global_threshold;
        TREQUIRE(q->global_stages >= 1 && q->global_coeffs, TETRIS_EINVAL, "query: global threshold without stages");
        TREQUIRE(g.ncomp == 2 && (int)g.level <= L && g.data && g.scale > 0, TETRIS_EINVAL,
                 "query: bad global threshold ciphertext");
        s.g_level = g.level;
        s.g_scale = g.scale;
        for (uint32_t st = 0; st < q->global_stages; st++)
            s.gstages.push_back(std::vector<double>(q->global_coeffs + st * nco, q->global_coeffs + (st + 1) * nco));
    }
    return s;
}

std::vector<const tetris_ct_in *> query_inputs(const tetris_query *q) {
    std::vector<const tetris_ct_in *> ins;
    for (uint32_t j = 0; j < q->n_attrs; j++) ins.push_back(&q->w[j]);
    for (uint32_t k = 0; k <= q->f_degree; k++) ins.push_back(&q->f_coeffs[k]);
    ins.push_back(q->threshold);
    if (q->global_threshold) ins.push_back(q->global_threshold);
    return ins;
}

static Program &get_program(Ctx &C, uint32_t dbh, const QuerySpec &s) {
    auto it = C.dbs.find(dbh);
    TREQUIRE(it != C.dbs.end(), TETRIS_ENOTFOUND, "unknown database handle");
    const std::string key = s.key(dbh);
    auto pit = C.programs.find(key);
    if (pit == C.programs.end()) {
        auto prog = record_query(C, it->second, s);
        pit = C.programs.emplace(key, std::move(prog)).first;
    }
    return *pit->second;
}

void drop_programs_of_db(Ctx &C, uint32_t dbh) {
    const std::string pre = "q" + std::to_string(dbh) + ":";
    for (auto it = C.programs.begin(); it != C.programs.end();) {
        if (it->first.compare(0, pre.size(), pre) == 0) it = C.programs.erase(it);
        else ++it;
    }
}

void evaluate_query(Ctx &C, uint32_t dbh, const tetris_query *q, tetris_ct_out *out, cudaStream_t s, bool device) {
    auto it = C.dbs.find(dbh);
    TREQUIRE(it != C.dbs.end(), TETRIS_ENOTFOUND, "unknown database handle");
    TREQUIRE(out && out->data, TETRIS_EINVAL, "query: null output");
    QuerySpec spec = spec_of(C, it->second, q);
    Program &P = get_program(C, dbh, spec);
    TREQUIRE(out->cap_words >= P.out_words, TETRIS_EINVAL, "query: output buffer too small");
    const cudaMemcpyKind in_kind = device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const auto ins = query_inputs(q);
    TREQUIRE(ins.size() == P.in_slots.size(), TETRIS_EINVAL, "query: inputs do not match the program");
    std::vector<const void *> srcs;
    for (auto *c : ins) srcs.push_back(c->data);
    P.copy_inputs(srcs, in_kind, s);
    if (C.profile) P.run_profiled(s, C.stats);
    else if (C.use_graph) P.run_graph(s);
    else P.run(s);
    TCHECK_CUDA(cudaMemcpyAsync(out->data, P.out_base, P.out_words * 8,
                                device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    out->level = P.out_level;
    out->ncomp = P.out_comps;
    out->scale = P.out_scale;
    if (!device) TCHECK_CUDA(cudaStreamSynchronize(s));
}

// the residues of a sum over partitions, reduced: x mod q_i (x < 2^63)
void reduce_sum(Ctx &C, u64 *data, int level, int ncomp, cudaStream_t s) {
    TREQUIRE(data && level >= 0 && level <= C.L() && ncomp >= 1 && ncomp <= 3, TETRIS_EINVAL, "reduce_sum: bad shape");
    Program P;
    Rec R(C, P);
    std::vector<EwJob> jobs;
    for (int c = 0; c < ncomp; c++)
        for (int i = 0; i <= level; i++) {
            EwJob j{};
            j.op = EW_REDUCE;
            j.prime = i;
            j.a = j.dst = data + ((size_t)c * (level + 1) + i) * C.N;
            jobs.push_back(j);
        }
    R.ew(jobs);
    P.finalize();
    P.run(s);
    TCHECK_CUDA(cudaStreamSynchronize(s));
}

// Time the recorded query under each candidate schedule; keep the fastest.
void autotune(Ctx &C, uint32_t dbh, const tetris_query *q, int reps, std::vector<tetris_tune_entry> &out) {
    auto it = C.dbs.find(dbh);
    TREQUIRE(it != C.dbs.end(), TETRIS_ENOTFOUND, "unknown database handle");
    const int blocks = it->second.blocks;
    std::vector<int> bpls = {0};
    for (int b : {8, 4, 2, 1})
        if (b < blocks) bpls.push_back(b);
    const int saved_bpl = C.blocks_per_launch, saved_loge = C.nt.loge, saved_pers = C.persistent;
    double best = 1e300;
    int best_bpl = saved_bpl, best_loge = saved_loge, best_pers = saved_pers;
    std::string best_key;
    cudaEvent_t e0, e1;
    TCHECK_CUDA(cudaEventCreate(&e0));
    TCHECK_CUDA(cudaEventCreate(&e1));
    // (loge, persistent): radix-8 or radix-16 register groups, or persistent launches (radix 8)
    std::vector<std::pair<int, int>> kinds = {{3, 0}, {4, 0}};
    if (C.log_n >= 14 && C.log_n <= 16) kinds.push_back({3, 1});
    for (auto kd : kinds)
        for (int bpl : bpls) {
            const int loge = kd.first;
            C.blocks_per_launch = bpl;
            C.nt.loge = loge;
            C.persistent = kd.second;
            QuerySpec spec = spec_of(C, it->second, q);
            const std::string key = spec.key(dbh);
            Program &P = get_program(C, dbh, spec);
            const auto ins = query_inputs(q);
            for (size_t slot = 0; slot < ins.size(); slot++)
                P.in_slots[slot].copy_from(ins[slot]->data, cudaMemcpyHostToDevice, C.stream);
            P.run_graph(C.stream);
            TCHECK_CUDA(cudaEventRecord(e0, C.stream));
            for (int r = 0; r < reps; r++) P.run_graph(C.stream);
            TCHECK_CUDA(cudaEventRecord(e1, C.stream));
            TCHECK_CUDA(cudaEventSynchronize(e1));
            float ms = 0;
            TCHECK_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            out.push_back({bpl, loge, ms / reps, kd.second, 0});
            if (ms / reps < best) {
                if (!best_key.empty()) C.programs.erase(best_key);
                best = ms / reps;
                best_bpl = bpl;
                best_loge = loge;
                best_pers = kd.second;
                best_key = key;
            } else {
                C.programs.erase(key);  // keep only the winner's buffers
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    C.blocks_per_launch = best_bpl;
    C.nt.loge = best_loge;
    C.persistent = best_pers;
}

void plan_info(Ctx &C, uint32_t dbh, uint32_t degree, uint32_t stages, tetris_plan_info *out) {
    auto it = C.dbs.find(dbh);
    TREQUIRE(it != C.dbs.end(), TETRIS_ENOTFOUND, "unknown database handle");
    QuerySpec s;
    s.attrs = it->second.attrs;
    s.degree = degree;
    for (uint32_t k = 0; k <= degree; k++) {
        s.c_level.push_back(C.L());
        s.c_scale.push_back(C.scale);
    }
    s.t_level = C.L();
    s.t_scale = C.scale;
    for (uint32_t i = 0; i < stages; i++) s.stages.push_back({35.0 / 16, -35.0 / 16, 21.0 / 16, -5.0 / 16});  // f3
    s.bpl = C.blocks_per_launch;
    s.loge = C.nt.loge;
    QPlan pl = make_plan(C, it->second.records, degree, s.stages);
    Program &P = get_program(C, dbh, s);
    out->l_lin = pl.l_lin;
    out->l_d = pl.l_d;
    out->l_y = pl.l_y;
    out->l_u = pl.l_u;
    out->l_out = pl.l_out;
    out->l_ret = pl.l_ret;
    out->ragged = pl.ragged;
    out->relins = P.relins;
    out->rescales = P.rescales;
    out->rotations = P.rotations;
    out->kernel_launches = P.kernel_launches;
    out->pt_scale = C.pt_scale;
    out->mask_scale = pl.mask_scale;
    out->input_words = 0;
    for (auto &sl : P.in_slots) out->input_words += sl.words();
}

}  // namespace tetris
