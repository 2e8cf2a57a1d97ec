// bsd_dem.cpp -- text detector error model (DEM) reader: (H, A, p) for bsd_create.
//
// The decoding problem of App. A is the triple (H, A, p): one column per
// error mechanism, H its detectors, A its logical observables, p its
// probability.  A DEM in the common text format lists those mechanisms:
//
//   error(0.001) D0 D5 L1          a mechanism: probability, then targets
//   error(0.002) D3 ^ D7           '^' separates parts of one mechanism;
//                                  its effect is the XOR of all parts
//   detector(1, 2, 0) D4           declares a detector (coordinates ignored)
//   logical_observable L2          declares an observable
//   shift_detectors(0, 0, 1) 72    adds 72 to every later detector index
//   repeat 11 { ... }              the block, 11 times (blocks nest)
//   # comment                      to the end of the line
//
// Instruction names may carry a tag in brackets (error[tag](p) ...), which is
// ignored.  Columns are numbered in the order the mechanisms are met (repeat
// blocks expanded); M is one more than the largest detector index met (or
// declared), K likewise for observables.  A target listed twice in one
// mechanism cancels.  With BSD_DEM_MERGE, mechanisms with identical
// (detector, observable) sets are merged into one column with probability
// p1 (1 - p2) + p2 (1 - p1) (either one, not both, happens).
#include <algorithm>
#include <cctype>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "bsd.h"

struct bsd_dem {
    int32_t M = 0, N = 0, K = 0;
    std::vector<std::vector<int32_t>> dets;   // per column, ascending
    std::vector<std::vector<int32_t>> obs;    // per column, ascending
    std::vector<double> p;
};

namespace {

struct Cursor {
    const char* s;
    const char* end;
    int64_t line = 1;

    bool done() const { return s >= end; }
    // skip spaces, tabs and comments; stop at a newline
    void blank()
    {
        while (s < end) {
            if (*s == ' ' || *s == '\t' || *s == '\r') { ++s; continue; }
            if (*s == '#') { while (s < end && *s != '\n') ++s; continue; }
            break;
        }
    }
    // skip everything blank including newlines
    void space()
    {
        for (;;) {
            blank();
            if (s < end && *s == '\n') { ++s; ++line; continue; }
            break;
        }
    }
};

struct Stmt {
    std::string name;
    std::vector<double> args;                 // numbers in parentheses
    std::vector<std::string> targets;         // D<k>, L<k>, ^, plain integers
    std::vector<Stmt> block;                  // repeat body
    int64_t line = 0;
};

struct ParseError {
    int64_t line;
    int code;
};

bool parse_block(Cursor& c, std::vector<Stmt>& out, bool nested);

bool parse_stmt(Cursor& c, Stmt& st)
{
    st.line = c.line;
    const char* b = c.s;
    while (c.s < c.end && (std::isalnum((unsigned char)*c.s) || *c.s == '_')) ++c.s;
    st.name.assign(b, c.s);
    if (st.name.empty()) throw ParseError{c.line, BSD_ERR_INVALID_ARG};
    if (c.s < c.end && *c.s == '[') {        // tag: ignored
        while (c.s < c.end && *c.s != ']' && *c.s != '\n') ++c.s;
        if (c.s >= c.end || *c.s != ']') throw ParseError{c.line, BSD_ERR_INVALID_ARG};
        ++c.s;
    }
    if (c.s < c.end && *c.s == '(') {
        ++c.s;
        for (;;) {
            c.blank();
            char* e = nullptr;
            const double v = std::strtod(c.s, &e);
            if (e == c.s || e > c.end) throw ParseError{c.line, BSD_ERR_INVALID_ARG};
            st.args.push_back(v);
            c.s = e;
            c.blank();
            if (c.s < c.end && *c.s == ',') { ++c.s; continue; }
            if (c.s < c.end && *c.s == ')') { ++c.s; break; }
            throw ParseError{c.line, BSD_ERR_INVALID_ARG};
        }
    }
    for (;;) {
        c.blank();
        if (c.s >= c.end || *c.s == '\n' || *c.s == '}') break;
        if (*c.s == '{') {
            ++c.s;
            if (!parse_block(c, st.block, true)) throw ParseError{c.line, BSD_ERR_INVALID_ARG};
            break;
        }
        const char* t = c.s;
        while (c.s < c.end && !std::isspace((unsigned char)*c.s) && *c.s != '{' && *c.s != '}' && *c.s != '#') ++c.s;
        st.targets.emplace_back(t, c.s);
    }
    return true;
}

// statements until the end of the text (nested = false) or a closing brace
bool parse_block(Cursor& c, std::vector<Stmt>& out, bool nested)
{
    for (;;) {
        c.space();
        if (c.done()) return !nested;
        if (*c.s == '}') {
            if (!nested) throw ParseError{c.line, BSD_ERR_INVALID_ARG};
            ++c.s;
            return true;
        }
        Stmt st;
        parse_stmt(c, st);
        out.push_back(std::move(st));
    }
}

// a nonnegative integer token (an index or a count)
long long to_index(const std::string& t, size_t from, int64_t line)
{
    if (t.size() <= from) throw ParseError{line, BSD_ERR_INVALID_ARG};
    long long v = 0;
    for (size_t k = from; k < t.size(); ++k) {
        if (!std::isdigit((unsigned char)t[k])) throw ParseError{line, BSD_ERR_INVALID_ARG};
        v = v * 10 + (t[k] - '0');
        if (v > (1ll << 31) - 2) throw ParseError{line, BSD_ERR_UNSUPPORTED};
    }
    return v;
}

struct Builder {
    bsd_dem* d;
    long long max_det = -1, max_obs = -1;
    long long columns_limit = (1ll << 31) - 2;

    void run(const std::vector<Stmt>& prog, long long& shift)
    {
        for (const Stmt& st : prog) {
            if (st.name == "error") {
                if (st.args.size() != 1 || !(st.args[0] >= 0.0) || !(st.args[0] <= 1.0))
                    throw ParseError{st.line, BSD_ERR_INVALID_ARG};
                std::vector<long long> dv, ov;
                for (const std::string& t : st.targets) {
                    if (t == "^") continue;
                    if (t[0] == 'D') dv.push_back(shift + to_index(t, 1, st.line));
                    else if (t[0] == 'L') ov.push_back(to_index(t, 1, st.line));
                    else throw ParseError{st.line, BSD_ERR_INVALID_ARG};
                }
                add_column(dv, ov, st.args[0], st.line);
            } else if (st.name == "detector") {
                for (const std::string& t : st.targets) {
                    if (t[0] != 'D') throw ParseError{st.line, BSD_ERR_INVALID_ARG};
                    max_det = std::max(max_det, shift + to_index(t, 1, st.line));
                }
            } else if (st.name == "logical_observable") {
                for (const std::string& t : st.targets) {
                    if (t[0] != 'L') throw ParseError{st.line, BSD_ERR_INVALID_ARG};
                    max_obs = std::max(max_obs, to_index(t, 1, st.line));
                }
            } else if (st.name == "shift_detectors") {
                if (st.targets.size() != 1) throw ParseError{st.line, BSD_ERR_INVALID_ARG};
                shift += to_index(st.targets[0], 0, st.line);
                if (shift > (1ll << 31) - 2) throw ParseError{st.line, BSD_ERR_UNSUPPORTED};
            } else if (st.name == "repeat") {
                if (st.targets.size() != 1) throw ParseError{st.line, BSD_ERR_INVALID_ARG};
                const long long n = to_index(st.targets[0], 0, st.line);
                for (long long r = 0; r < n; ++r) run(st.block, shift);
            } else {
                throw ParseError{st.line, BSD_ERR_UNSUPPORTED};
            }
        }
    }

    void add_column(std::vector<long long>& dv, std::vector<long long>& ov, double p, int64_t line)
    {
        // a target met twice cancels (the effect is the XOR of all parts)
        auto xor_reduce = [](std::vector<long long>& v) {
            std::sort(v.begin(), v.end());
            std::vector<long long> r;
            for (size_t k = 0; k < v.size();) {
                size_t k2 = k;
                while (k2 < v.size() && v[k2] == v[k]) ++k2;
                if ((k2 - k) & 1) r.push_back(v[k]);
                k = k2;
            }
            v.swap(r);
        };
        xor_reduce(dv);
        xor_reduce(ov);
        if ((long long)d->p.size() >= columns_limit) throw ParseError{line, BSD_ERR_UNSUPPORTED};
        for (long long x : dv) max_det = std::max(max_det, x);
        for (long long x : ov) max_obs = std::max(max_obs, x);
        d->dets.emplace_back(dv.begin(), dv.end());
        d->obs.emplace_back(ov.begin(), ov.end());
        d->p.push_back(p);
    }
};

void merge_identical(bsd_dem* d)
{
    std::map<std::pair<std::vector<int32_t>, std::vector<int32_t>>, size_t> first;
    std::vector<std::vector<int32_t>> dets, obs;
    std::vector<double> p;
    for (size_t j = 0; j < d->p.size(); ++j) {
        auto key = std::make_pair(d->dets[j], d->obs[j]);
        auto it = first.find(key);
        if (it == first.end()) {
            first.emplace(std::move(key), p.size());
            dets.push_back(d->dets[j]);
            obs.push_back(d->obs[j]);
            p.push_back(d->p[j]);
        } else {
            const double a = p[it->second], b = d->p[j];
            p[it->second] = a * (1.0 - b) + b * (1.0 - a);
        }
    }
    d->dets.swap(dets);
    d->obs.swap(obs);
    d->p.swap(p);
}

}  // namespace

extern "C" {

int bsd_dem_parse(const char* text, int64_t len, int32_t flags, bsd_dem** out, int64_t* err_line)
{
    if (err_line) *err_line = 0;
    if (!text || len < 0 || !out || (flags & ~BSD_DEM_MERGE)) return BSD_ERR_INVALID_ARG;
    *out = nullptr;
    bsd_dem* d = new (std::nothrow) bsd_dem;
    if (!d) return BSD_ERR_OOM;
    try {
        const std::string buf(text, (size_t)len);   // NUL-terminated copy for the number parser
        Cursor c{buf.c_str(), buf.c_str() + buf.size()};
        std::vector<Stmt> prog;
        parse_block(c, prog, false);
        Builder b{d};
        long long shift = 0;
        b.run(prog, shift);
        if (flags & BSD_DEM_MERGE) merge_identical(d);
        d->M = (int32_t)(b.max_det + 1);
        d->K = (int32_t)(b.max_obs + 1);
        d->N = (int32_t)d->p.size();
    } catch (const ParseError& e) {
        if (err_line) *err_line = e.line;
        delete d;
        return e.code;
    } catch (const std::bad_alloc&) {
        delete d;
        return BSD_ERR_OOM;
    }
    *out = d;
    return BSD_OK;
}

int bsd_dem_sizes(const bsd_dem* dem, int32_t* M, int32_t* N, int32_t* K, int64_t* nnz_H, int64_t* nnz_A)
{
    if (!dem) return BSD_ERR_INVALID_ARG;
    int64_t h = 0, a = 0;
    for (size_t j = 0; j < dem->p.size(); ++j) {
        h += (int64_t)dem->dets[j].size();
        a += (int64_t)dem->obs[j].size();
    }
    if (M) *M = dem->M;
    if (N) *N = dem->N;
    if (K) *K = dem->K;
    if (nnz_H) *nnz_H = h;
    if (nnz_A) *nnz_A = a;
    return BSD_OK;
}

int bsd_dem_fill(const bsd_dem* dem, int32_t* H_row_ptr, int32_t* H_col_idx, int32_t* A_row_ptr, int32_t* A_col_idx,
                 double* priors)
{
    if (!dem || !H_row_ptr || !H_col_idx || !A_row_ptr || !priors || (dem->K > 0 && !A_col_idx))
        return BSD_ERR_INVALID_ARG;
    // CSR by rows: count, prefix, then fill scanning columns in order, so the
    // column indices of every row come out ascending
    auto csr = [&](const std::vector<std::vector<int32_t>>& cols, int32_t rows, int32_t* rp, int32_t* ci) {
        std::vector<int64_t> cnt((size_t)rows + 1, 0);
        for (const auto& c : cols)
            for (int32_t r : c) cnt[(size_t)r + 1]++;
        for (int32_t r = 0; r < rows; ++r) cnt[(size_t)r + 1] += cnt[(size_t)r];
        for (int32_t r = 0; r <= rows; ++r) rp[r] = (int32_t)cnt[(size_t)r];
        std::vector<int64_t> fill(cnt.begin(), cnt.end() - 1);
        for (size_t j = 0; j < cols.size(); ++j)
            for (int32_t r : cols[j]) ci[fill[(size_t)r]++] = (int32_t)j;
    };
    csr(dem->dets, dem->M, H_row_ptr, H_col_idx);
    csr(dem->obs, dem->K, A_row_ptr, A_col_idx);
    for (size_t j = 0; j < dem->p.size(); ++j) priors[j] = dem->p[j];
    return BSD_OK;
}

void bsd_dem_free(bsd_dem* dem) { delete dem; }

}  // extern "C"
