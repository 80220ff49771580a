"""Host build of the double-float helpers that the mixed form's defect
correction runs on the GPU (paper_0710_0736_gb300/csrc/ac_df64.cuh): the
integer-pipe binary64 <-> binary32 conversions and the binary64 split are
checked against numpy's IEEE conversions and exact rational arithmetic, the
error-free transformations against exact sums and products, and the mixed
form's node update u <- P_G(u + delta) (float kept set, binary64 theta)
against the plain binary64 iteration and a sort-based simplex projection."""
import os
import shutil
import subprocess
from fractions import Fraction

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_0710_0736_gb300", "csrc")

HARNESS = r"""
#include "ac_df64.cuh"
#include <cstdio>
#include <cstring>
#include <cstdlib>
#include <vector>
// records of (N doubles u, N floats delta) -> (u' by outer_update_node, its
// path as a double, u' by the binary64-only iteration)
template <int N>
void update_records(const std::vector<unsigned char> &in) {
  const size_t rec = 12 * N;
  const size_t n = in.size() / rec;
  for (size_t i = 0; i < n; ++i) {
    double u[N], v[N];
    float d[N];
    std::memcpy(u, &in[rec * i], 8 * N);
    std::memcpy(d, &in[rec * i + 8 * N], 4 * N);
    std::memcpy(v, u, 8 * N);
    auto id = [](unsigned m) { return m; };
    const double p = ac::outer_update_node<N>(u, d, id);
    ac::outer_update_node<N, true>(v, d, id);
    fwrite(u, 8, N, stdout);
    fwrite(&p, 8, 1, stdout);
    fwrite(v, 8, N, stdout);
  }
}
int main(int argc, char **argv) {
  std::vector<unsigned char> in;
  unsigned char buf[1 << 16];
  size_t k;
  while ((k = fread(buf, 1, sizeof buf, stdin)) > 0) in.insert(in.end(), buf, buf + k);
  const char mode = argv[1][0];
  if (mode == 'd') {  // doubles -> (rn, h, l) floats
    size_t n = in.size() / 8;
    for (size_t i = 0; i < n; ++i) {
      double d;
      std::memcpy(&d, &in[8 * i], 8);
      float o[3];
      o[0] = ac::f64_to_f32_rn(d);
      ac::split_f64(d, o[1], o[2]);
      fwrite(o, 4, 3, stdout);
    }
  } else if (mode == 'f') {  // floats -> doubles
    size_t n = in.size() / 4;
    for (size_t i = 0; i < n; ++i) {
      float f;
      std::memcpy(&f, &in[4 * i], 4);
      double d = ac::f32_to_f64(f);
      fwrite(&d, 8, 1, stdout);
    }
  } else if (mode == 'h') {  // doubles -> f64_head
    size_t n = in.size() / 8;
    for (size_t i = 0; i < n; ++i) {
      double d;
      std::memcpy(&d, &in[8 * i], 8);
      float o = ac::f64_head(d);
      fwrite(&o, 4, 1, stdout);
    }
  } else if (mode == 'u') {  // node updates, N from argv[2]
    switch (argc > 2 ? std::atoi(argv[2]) : 8) {
      case 2: update_records<2>(in); break;
      case 3: update_records<3>(in); break;
      case 5: update_records<5>(in); break;
      default: update_records<8>(in); break;
    }
  } else if (mode == 'a') {  // float quadruples (ah, al, bh, bl) -> add_f2
    size_t n = in.size() / 16;
    for (size_t i = 0; i < n; ++i) {
      float q[4];
      std::memcpy(q, &in[16 * i], 16);
      ac::f2 r = ac::add_f2({q[0], q[1]}, q[2], q[3]);
      fwrite(&r, 4, 2, stdout);
    }
  } else {  // float quadruples (a, b, c, d) -> two_sum(a, b), fast_two_sum(a, b), (a + c)(b + d)
    size_t n = in.size() / 16;
    for (size_t i = 0; i < n; ++i) {
      float q[4];
      std::memcpy(q, &in[16 * i], 16);
      ac::f2 s = ac::two_sum(q[0], q[1]), f = ac::fast_two_sum(q[0], q[1]), m = ac::mul_f2(q[0], q[2], q[1], q[3]);
      float o[6] = {s.h, s.l, f.h, f.l, m.h, m.l};
      fwrite(o, 4, 6, stdout);
    }
  }
  return 0;
}
"""


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no C++ compiler")
    d = tmp_path_factory.mktemp("df64")
    src = d / "h.cpp"
    src.write_text(HARNESS)
    exe = d / "h"
    subprocess.run([cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-I", CSRC, str(src), "-o", str(exe)], check=True)

    def run(mode, arr, *extra):
        out = subprocess.run([str(exe), mode, *extra], input=np.ascontiguousarray(arr).tobytes(),
                             capture_output=True, check=True).stdout
        return out

    return run


def _doubles(rng, n):
    e = rng.integers(-150, 140, n).astype(np.float64)
    m = rng.random(n) + 1.0
    d = np.ldexp(m, e.astype(np.int64)) * rng.choice([-1.0, 1.0], n)
    bits = rng.integers(0, 2**63, n, dtype=np.uint64) | (rng.integers(0, 2, n, dtype=np.uint64) << np.uint64(63))
    d2 = bits.view(np.float64)
    d2 = d2[np.isfinite(d2) & (np.abs(d2) < 2.0**140) & (np.abs(d2) > 2.0**-150)]
    special = [0.0, -0.0, 1.0, -1.0, 0.5, 1.0 / 3.0, 2.0**-126, -(2.0**-126), np.nextafter(2.0**-126, 0),
               2.0**-97, np.nextafter(2.0**-97, 0), 2.0**-96, float(np.finfo(np.float32).max),
               np.nextafter(2.0**128, 0), 2.0**128, -(2.0**130), np.inf, -np.inf, np.nan, 1e-300, -1e300]
    # exact ties and near-ties of the binary32 rounding: 29 dropped bits 1000...0, 1000...1, 0111...1
    base = np.frombuffer(np.array([1.0, 1.5, 0.75, 3.0 + 2.0**-22], dtype=np.float64).tobytes(), dtype=np.uint64)
    ties = []
    for b in base:
        for low in (0x10000000, 0x10000001, 0x0FFFFFFF, 0x30000000, 0x1FFFFFFF):
            v = (int(b) & ~0x1FFFFFFF) | low
            ties.append(np.array([v], dtype=np.uint64).view(np.float64)[0])
            ties.append(np.array([v | (1 << 29)], dtype=np.uint64).view(np.float64)[0])
    return np.concatenate([d, d2, np.array(special), np.array(ties), -np.array(ties)])


def test_narrow_matches_ieee_rounding(harness):
    rng = np.random.default_rng(5)
    d = _doubles(rng, 20000)
    out = np.frombuffer(harness("d", d), dtype=np.float32).reshape(-1, 3)
    rn = out[:, 0]
    a = np.abs(d)
    normal = (a >= 2.0**-126) & (a < 2.0**128)
    with np.errstate(over="ignore"):
        ref = d.astype(np.float32)
    assert (rn[normal].view(np.uint32) == ref[normal].view(np.uint32)).all()
    tiny = a < 2.0**-126
    assert (rn[tiny] == 0).all() and (np.signbit(rn[tiny]) == np.signbit(d[tiny])).all()
    big = np.isfinite(d) & (a >= 2.0**128)
    assert np.isinf(rn[big]).all() and (np.sign(rn[big]) == np.sign(d[big])).all()
    assert np.isnan(rn[np.isnan(d)]).all()
    assert (np.isinf(rn[np.isinf(d)]) & (np.sign(rn[np.isinf(d)]) == np.sign(d[np.isinf(d)]))).all()


def test_split_is_truncation_plus_tail(harness):
    rng = np.random.default_rng(6)
    d = _doubles(rng, 20000)
    out = np.frombuffer(harness("d", d), dtype=np.float32).reshape(-1, 3)
    h, l = out[:, 1], out[:, 2]
    a = np.abs(d)
    normal = np.isfinite(d) & (a >= 2.0**-126) & (a < 2.0**128)
    # the head is the significand truncated to 24 bits
    bits = d.view(np.uint64)
    ah = (bits >> np.uint64(32)).astype(np.uint64) & np.uint64(0x7FFFFFFF)
    lo = bits & np.uint64(0xFFFFFFFF)
    t = (((ah - np.uint64(0x38000000)) << np.uint64(3)) & np.uint64(0xFFFFFFFF)) | (lo >> np.uint64(29))
    assert (h[normal].view(np.uint32) & np.uint32(0x7FFFFFFF) == t[normal].astype(np.uint32)).all()
    assert (np.signbit(h[normal]) == np.signbit(d[normal])).all()
    for i in np.flatnonzero(normal):
        err = abs(Fraction(float(d[i])) - Fraction(float(h[i])) - Fraction(float(l[i])))
        if a[i] >= 2.0**-97:
            assert err <= Fraction(float(a[i])) / 2**47, (d[i], h[i], l[i])
            assert l[i] == 0 or np.signbit(l[i]) == np.signbit(d[i])
        else:
            assert l[i] == 0 and err < Fraction(float(a[i])) / 2**23
    tiny = a < 2.0**-126
    assert (h[tiny] == 0).all() and (l[tiny] == 0).all()
    assert np.isnan(h[np.isnan(d)]).all() and (l[~np.isfinite(d)] == 0).all()
    assert np.isinf(h[np.isinf(d)]).all()


def test_widen_is_exact(harness):
    rng = np.random.default_rng(7)
    f = rng.integers(0, 2**32, 20000, dtype=np.uint64).astype(np.uint32).view(np.float32)
    f = np.concatenate([f, np.array([0.0, -0.0, 1.0, np.inf, -np.inf, np.nan, 1e-40, -1e-45,
                                     np.finfo(np.float32).tiny, np.finfo(np.float32).max], dtype=np.float32)])
    got = np.frombuffer(harness("f", f), dtype=np.float64)
    normal = np.isfinite(f) & (np.abs(f) >= np.finfo(np.float32).tiny)
    assert (got[normal] == f[normal].astype(np.float64)).all()
    sub = np.isfinite(f) & (np.abs(f) < np.finfo(np.float32).tiny)
    assert (got[sub] == 0).all() and (np.signbit(got[sub]) == np.signbit(f[sub])).all()
    assert np.isnan(got[np.isnan(f)]).all()
    assert (got[np.isinf(f)] == f[np.isinf(f)].astype(np.float64)).all()


def test_error_free_transformations(harness):
    rng = np.random.default_rng(8)
    n = 4000
    a = (rng.standard_normal(n) * np.exp2(rng.integers(-30, 30, n))).astype(np.float32)
    b = (rng.standard_normal(n) * np.exp2(rng.integers(-30, 30, n))).astype(np.float32)
    # |a| >= |b| for the fast two-sum: order each pair
    swap = np.abs(a) < np.abs(b)
    a2, b2 = np.where(swap, b, a), np.where(swap, a, b)
    # tails below half an ulp of their heads: (a2 + c, b2 + dd) are double-floats
    c = (a2 * rng.random(n).astype(np.float32) * np.float32(2.0**-25)).astype(np.float32)
    dd = (b2 * rng.random(n).astype(np.float32) * np.float32(2.0**-25)).astype(np.float32)
    q = np.stack([a2, b2, c, dd], 1).astype(np.float32)
    out = np.frombuffer(harness("s", q), dtype=np.float32).reshape(-1, 6)
    for i in range(n):
        x, y = Fraction(float(q[i, 0])), Fraction(float(q[i, 1]))
        assert Fraction(float(out[i, 0])) + Fraction(float(out[i, 1])) == x + y
        assert Fraction(float(out[i, 2])) + Fraction(float(out[i, 3])) == x + y
        prod = (x + Fraction(float(q[i, 2]))) * (y + Fraction(float(q[i, 3])))
        got = Fraction(float(out[i, 4])) + Fraction(float(out[i, 5]))
        assert abs(got - prod) <= abs(prod) / 2**44


def test_double_float_add(harness):
    rng = np.random.default_rng(9)
    n = 4000
    ah = (rng.standard_normal(n) * np.exp2(rng.integers(-20, 20, n))).astype(np.float32)
    bh = (rng.standard_normal(n) * np.exp2(rng.integers(-20, 20, n))).astype(np.float32)
    bh[: n // 4] = -ah[: n // 4] * np.float32(1 + 2.0**-20)  # near-cancellation
    al = (ah * rng.uniform(-1, 1, n).astype(np.float32) * np.float32(2.0**-25)).astype(np.float32)
    bl = (bh * rng.uniform(-1, 1, n).astype(np.float32) * np.float32(2.0**-25)).astype(np.float32)
    q = np.stack([ah, al, bh, bl], 1).astype(np.float32)
    out = np.frombuffer(harness("a", q), dtype=np.float32).reshape(-1, 2)
    for i in range(n):
        a = Fraction(float(q[i, 0])) + Fraction(float(q[i, 1]))
        b = Fraction(float(q[i, 2])) + Fraction(float(q[i, 3]))
        got = Fraction(float(out[i, 0])) + Fraction(float(out[i, 1]))
        assert abs(got - (a + b)) <= (abs(a) + abs(b)) / 2**46
        # renormalised: the tail is below one ulp of the head
        assert abs(float(out[i, 1])) <= abs(float(out[i, 0])) * 2.0**-23


def test_head_is_the_truncated_significand(harness):
    """f64_head (the pixel-label filter's conversion) is split_f64's head:
    the significand truncated to 24 bits, 0 below 2^-126, NaN from 2^128."""
    rng = np.random.default_rng(10)
    d = _doubles(rng, 20000)
    head = np.frombuffer(harness("h", d), dtype=np.float32)
    h = np.frombuffer(harness("d", d), dtype=np.float32).reshape(-1, 3)[:, 1]
    a = np.abs(d)
    normal = np.isfinite(d) & (a >= 2.0**-126) & (a < 2.0**128)
    assert (head[normal].view(np.uint32) == h[normal].view(np.uint32)).all()
    # and the numpy restatement the node-update test uses
    assert (_head32(d[normal]).view(np.uint32) == head[normal].view(np.uint32)).all()
    assert (head[a < 2.0**-126] == 0).all()
    assert np.isnan(head[~np.isfinite(d) | (a >= 2.0**128)]).all()
    for i in np.flatnonzero(normal)[:4000]:
        assert abs(Fraction(float(d[i])) - Fraction(float(head[i]))) <= Fraction(float(a[i])) / 2**23


def _filter_sums(head, U):
    """The label filter's float sums, in the kernel's order: 2 h00, + h10,
    + h01, + 2 h11 (float32 arithmetic)."""
    h = lambda q: np.frombuffer(head(np.ascontiguousarray(q)), dtype=np.float32).reshape(q.shape)
    v = np.float32(2) * h(U[0])
    v = v + h(U[1])
    v = v + h(U[2])
    return v + np.float32(2) * h(U[3])


def test_pixel_label_filter_bound(harness):
    """The pixel-label filter (Sec. 4.3 labels; k_pixel_labels): for phase
    values in [0, 1] its float sums are within 1.5e-6 of the exact
    2 u00 + u10 + u01 + 2 u11, so a float lead above 4e-6 fixes the argmax
    of the binary64 sums.  Checked on random values, values just below
    powers of two (the largest truncation errors) and exact ties."""
    rng = np.random.default_rng(11)
    n = 3000
    U = rng.random((4, n))
    # largest truncation error: significands 1.111...1 just below 1, 1/2, 1/4
    below = np.array([np.nextafter(2.0**-k, 0) for k in range(0, 4)])
    U[:, : 4 * 200] = np.repeat(below, 200)[None, :] * (1 - rng.random((4, 800)) * 2.0**-30)
    U[:, 900:1000] = 1.0
    U[:, 1000:1100] = 0.0
    v = _filter_sums(lambda q: harness("h", q), U).astype(np.float64)
    for i in range(n):
        exact = 2 * Fraction(float(U[0, i])) + Fraction(float(U[1, i])) + Fraction(float(U[2, i])) \
            + 2 * Fraction(float(U[3, i]))
        assert abs(Fraction(float(v[i])) - exact) < Fraction(3, 2 * 10**6), (U[:, i], v[i])
    # two phases per pixel: where the float lead exceeds 4e-6 the binary64
    # sums order the phases the same way
    a = rng.random((4, n))
    b = np.clip(a + rng.choice([0.0, 1e-9, -1e-9, 3e-7, -3e-7, 1e-6, -1e-6, 5e-6, -5e-6], (4, n)), 0, 1)
    va = _filter_sums(lambda q: harness("h", q), a)
    vb = _filter_sums(lambda q: harness("h", q), b)
    sa = 2 * a[0] + a[1] + a[2] + 2 * a[3]
    sb = 2 * b[0] + b[1] + b[2] + 2 * b[3]
    lead = (va - vb).astype(np.float64)
    sure = np.abs(lead) > 4e-6
    assert sure.any() and (~sure).any()
    assert (np.sign(lead[sure]) == np.sign(sa[sure] - sb[sure])).all()


def _proj_simplex_sort(v):
    """Euclidean projection onto {x >= 0, sum x = 1} by sorting (the
    textbook rule: theta from the largest prefix whose mean-shifted entries
    stay positive), independent of Michelot's iteration."""
    s = np.sort(v)[::-1]
    c = np.cumsum(s) - 1.0
    k = np.arange(1, len(v) + 1)
    rho = np.nonzero(s - c / k > 0)[0][-1]
    return np.maximum(v - c[rho] / (rho + 1), 0.0)


def _head32(x):
    """f64_head written with numpy: the binary64 significand cut to 24 bits
    (exact in binary32), a signed zero below 2^-126."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    h = (x.view(np.uint64) & ~np.uint64((1 << 29) - 1)).view(np.float64).astype(np.float32)
    tiny = np.abs(x) < 2.0**-126
    h[tiny] = np.copysign(np.float32(0), x[tiny]).astype(np.float32)
    return h


def _update_cases(rng, n, N):
    """Records (u, delta) of the mixed form's outer update: u on the
    simplex with exact zeros, delta float corrections, some components put on
    their bound (delta_i = -head(u_i), the float obstacle); then near ties, where an updated
    component lies within 1e-17 .. 1e-5 of the final threshold."""
    u = rng.dirichlet(np.full(N, 0.7), n)
    u[rng.random((n, N)) < 0.3] = 0.0
    u[np.arange(n), rng.integers(0, N, n)] += 0.05
    u /= u.sum(1, keepdims=True)
    d = (rng.standard_normal((n, N)) * 10.0 ** rng.uniform(-6, -1, (n, 1))).astype(np.float32)
    bound = rng.random((n, N)) < 0.25
    d[bound] = -_head32(u[bound])
    # near ties: final support K, threshold t, the others just below t
    m = n // 2
    p = rng.dirichlet(np.ones(N), m)
    p[rng.random((m, N)) < 0.4] = 0.0
    p[np.arange(m), rng.integers(0, N, m)] += 0.1
    p /= p.sum(1, keepdims=True)
    t = rng.uniform(-0.05, 0.05, (m, 1))
    gap = 10.0 ** rng.uniform(-17, -5, (m, N)) * rng.choice([0.0, 1.0], (m, N), p=[0.2, 0.8])
    v = np.where(p > 0, p + t, t - gap)
    dt = (rng.standard_normal((m, N)) * 1e-3).astype(np.float32)
    ut = v - dt.astype(np.float64)
    u = np.concatenate([u, ut, np.zeros((1, N)), np.full((1, N), 0.125)])
    d = np.concatenate([d, dt, np.zeros((1, N), np.float32), -np.full((1, N), 0.125, np.float32)])
    return u, d


@pytest.mark.parametrize("N,n", [(8, 40000), (5, 20000), (3, 20000), (2, 20000)])
def test_outer_update_node(harness, N, n):
    rng = np.random.default_rng(11 + N)
    u, d = _update_cases(rng, n, N)
    rec = np.concatenate([u.view(np.uint8).reshape(len(u), 8 * N), d.view(np.uint8).reshape(len(d), 4 * N)], axis=1)
    out = np.frombuffer(harness("u", rec, str(N)), dtype=np.float64).reshape(-1, 2 * N + 1)
    fast, path, plain = out[:, :N], out[:, N], out[:, N + 1:]
    # bit-identical to the binary64 iteration, whichever path ran
    assert (fast.view(np.uint64) == plain.view(np.uint64)).all()
    # the float set is accepted at all but near-tie nodes (rows with every
    # component on its bound take path 2); the near ties take both paths
    live = path[:n] != 2
    assert (path[:n][live] == 0).mean() > 0.99
    assert (fast[:n][~live] == 0).all()
    assert (path[n:-2] == 0).sum() > n // 40 and (path[n:-2] == 1).sum() > n // 40
    # the all-bound record: no kept component, u zeroed for the caller's projection
    assert path[-1] == 2 and (fast[-1] == 0).all()
    # against the sort-based projection of v = u + delta over the kept
    # components (the bound ones exactly 0)
    keep = d != -_head32(u)
    v = u + d.astype(np.float64)
    worst = 0.0
    for i in range(len(u) - 1):
        if not keep[i].any():
            continue
        x = np.zeros(N)
        x[keep[i]] = _proj_simplex_sort(v[i][keep[i]])
        worst = max(worst, np.abs(x - fast[i]).max())
        assert (fast[i][~keep[i]] == 0).all() and (fast[i] >= 0).all()
    assert worst < 1e-15, worst
