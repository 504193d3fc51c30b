"""Mutation check of the oracle's pins (opt-in: DP_ORACLE_MUTATIONS=1; about
fifteen minutes).  Each case plants one plausible mistake -- a dropped term, a
wrong sign or index, a swapped operand, a tie rule turned round -- in a copy of
oracle/ in a temporary directory, builds that copy, and runs the CPU suite
against it (the copy first on the import path).  Every case must make some
pin fail.  The committed oracle is never modified.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

pytestmark = pytest.mark.mutation

# (file in oracle/, what the mistake is, the text it replaces, the mistaken text)
MUTATIONS = [
 ("dp_oracle.c", "orbit centrifugal sign", "f[1] = vt * vt / r - p->mu / (r * r) + am * sin(alpha);", "f[1] = -vt * vt / r - p->mu / (r * r) + am * sin(alpha);"),
 ("dp_oracle.c", "orbit gravity 1/r^3", "- p->mu / (r * r) + am * sin(alpha);", "- p->mu / (r * r * r) + am * sin(alpha);"),
 ("dp_oracle.c", "orbit thrust radial cos", "+ am * sin(alpha);", "+ am * cos(alpha);"),
 ("dp_oracle.c", "orbit coupling sign", "f[2] = -vr * vt / r + am * cos(alpha);", "f[2] = vr * vt / r + am * cos(alpha);"),
 ("dp_oracle.c", "mass rate sign", "f[3] = -p->accel / p->exhaust_c;", "f[3] = p->accel / p->exhaust_c;"),
 ("dp_oracle.c", "a times m", "double am = p->accel / m;", "double am = p->accel * m;"),
 ("dp_oracle.c", "polar centrifugal sign", "f[1] = vt * vt / r - p->mu / (r * r) + u * sa;", "f[1] = -vt * vt / r - p->mu / (r * r) + u * sa;"),
 ("dp_oracle.c", "polar theta rate", "f[3] = vt / r;", "f[3] = vr / r;"),
 ("dp_oracle.c", "polar thrust swap", "+ u * sa;", "+ u * ca;"),
 ("dp_oracle.c", "polar coupling dropped", "f[2] = -vr * vt / r + u * ca;", "f[2] = u * ca;"),
 ("dp_oracle.c", "heun k2 only", "delta[d] = 0.5 * h * (k1[d] + k2[d]);", "delta[d] = h * k2[d];"),
 ("dp_oracle.c", "heun half predictor", "xt[d] = x[d] + h * k1[d];", "xt[d] = x[d] + 0.5 * h * k1[d];"),
 ("dp_oracle.c", "rk4 weights", "(k1[d] + 2.0 * k2[d] + 2.0 * k3[d] + k4[d])", "(k1[d] + 2.0 * k2[d] + k3[d] + 2.0 * k4[d])"),
 ("dp_oracle.c", "rk4 stage 4 from k2", "y[d] = x[d] + h * k3[d];", "y[d] = x[d] + h * k2[d];"),
 ("dp_oracle.c", "drag radial sign", "f[1] -= drag_c * x[1] * x[1];", "f[1] += drag_c * x[1] * x[1];"),
 ("dp_oracle.c", "drag transverse wrong comp", "f[2] -= drag_c * x[2] * x[2];", "f[2] -= drag_c * x[1] * x[2];"),
 ("dp_oracle.c", "interp weights swapped", "w *= bit ? t[d] : 1.0 - t[d];", "w *= bit ? 1.0 - t[d] : t[d];"),
 ("dp_oracle.c", "interp strict upper edge", "if (!(s[d] >= 0.0 && s[d] <= (double)(p->n[d] - 1))) return 0;", "if (!(s[d] >= 0.0 && s[d] < (double)(p->n[d] - 1))) return 0;"),
 ("dp_oracle.c", "q drops beta", "return p->dt * orc_running_cost(p, x, !isnan(alpha)) + p->beta * I;", "return p->dt * orc_running_cost(p, x, !isnan(alpha)) + I;"),
 ("dp_oracle.c", "q drops dt on cost", "return p->dt * orc_running_cost(p, x, !isnan(alpha)) + p->beta * I;", "return orc_running_cost(p, x, !isnan(alpha)) + p->beta * I;"),
 ("dp_oracle.c", "q grid units multiply", "    for (int d = 0; d < 4; ++d) s[d] = idx[d] + delta[d] / spacing(p, d);\n    if (!orc_interp(p, V, active, s, &I)) I = p->M;\n    return p->dt", "    for (int d = 0; d < 4; ++d) s[d] = idx[d] + delta[d] * spacing(p, d);\n    if (!orc_interp(p, V, active, s, &I)) I = p->M;\n    return p->dt"),
 ("dp_oracle.c", "penalty zero", "    if (!orc_interp(p, V, active, s, &I)) I = p->M;\n    return p->dt", "    if (!orc_interp(p, V, active, s, &I)) I = 0.0;\n    return p->dt"),
 ("dp_oracle.c", "q_state discount beta", "pow(p->beta, tau / p->dt) * I", "p->beta * I"),
 ("dp_oracle.c", "q_state cost dt", "return tau * orc_running_cost(p, y, !isnan(alpha))", "return p->dt * orc_running_cost(p, y, !isnan(alpha))"),
 ("dp_oracle.c", "q_state no lo shift", "s[d] = (y[d] + delta[d] - p->lo[d]) / spacing(p, d);", "s[d] = (y[d] + delta[d]) / spacing(p, d);"),
 ("dp_oracle.c", "energy 1/r^2", "return 0.5 * (x[1] * x[1] + x[2] * x[2]) - p->mu / x[0];", "return 0.5 * (x[1] * x[1] + x[2] * x[2]) - p->mu / (x[0] * x[0]);"),
 ("dp_oracle.c", "energy drops v_r", "return 0.5 * (x[1] * x[1] + x[2] * x[2]) - p->mu / x[0];", "return 0.5 * (x[2] * x[2]) - p->mu / x[0];"),
 ("dp_oracle.c", "band upper bound dropped", "return e >= p->e_lo && e <= p->e_hi;", "return e >= p->e_lo;"),
 ("dp_oracle.c", "vis-viva factor", "*a = p->mu * r / (2.0 * p->mu - r * v2);", "*a = p->mu * r / (p->mu - r * v2);"),
 ("dp_oracle.c", "e transverse sign", "double et = -r * vr * vt / p->mu;", "double et = r * vr * vt / p->mu;"),
 ("dp_oracle.c", "e rotation sign", "*ex = er * cos(th) - et * sin(th);", "*ex = er * cos(th) + et * sin(th);"),
 ("dp_oracle.c", "cost a linear", "p->cost_beta * (a - p->a_bar) * (a - p->a_bar)", "p->cost_beta * (a - p->a_bar)"),
 ("dp_oracle.c", "cost alpha no accel", "p->cost_alpha * (thrust_on ? p->accel : 0.0)", "p->cost_alpha * (thrust_on ? 1.0 : 0.0)"),
 ("dp_oracle.c", "enumerate ties high", "        if (q < qb) { qb = q; kb = k; }", "        if (q <= qb) { qb = q; kb = k; }"),
 ("dp_oracle.c", "walk one step only", "for (int step = 0; step < K; ++step) {", "for (int step = 0; step < 1; ++step) {"),
 ("dp_oracle.c", "walk never left", "if (ql < qk && ql <= qr) { k = kl; qk = ql; }", "if (0) { k = kl; qk = ql; }"),
 ("dp_oracle.c", "fib stops early", "for (int kk = n; kk > 4 && F[kk] * step_rad > p->refine_tol; --kk) {", "for (int kk = n; kk > 6 && F[kk] * step_rad > p->refine_tol; --kk) {"),
 ("dp_oracle.c", "fib wrong index", "            x1 = a + F[kk - 3];", "            x1 = a + F[kk - 2];"),
 ("dp_oracle.c", "fib right half only", "long lo_off = cl - ck, hi_off = cr - ck, L = hi_off - lo_off;", "long lo_off = 0, hi_off = cr - ck, L = hi_off - lo_off;"),
 ("dp_oracle.c", "fib not best kept", "    long best = ck;\n    double qb = qk;", "    long best = ck;\n    double qb = INFINITY;"),
 ("dp_oracle.c", "off control loses ties", "        if (q_off <= q) { q = q_off; code = ORC_CODE_OFF; }\n    }\n    *v_out = q;", "        if (q_off < q) { q = q_off; code = ORC_CODE_OFF; }\n    }\n    *v_out = q;"),
 ("dp_oracle.c", "residual signed", "        double dv = fabs(v - V_in[j]);", "        double dv = v - V_in[j];"),
 ("dp_oracle.c", "PI walks first", "int mode = (outer == 0 || !walk) ? ORC_IMPROVE_FULL : ORC_IMPROVE_WALK;", "int mode = walk ? ORC_IMPROVE_WALK : ORC_IMPROVE_FULL;"),
 ("dp_oracle.c", "vi diag drops beta on self", "q = (p->dt + p->beta * rest) / (1.0 - p->beta * self);", "q = (p->dt + p->beta * rest) / (1.0 - self);"),
 ("dp_oracle.c", "policy row penalty no beta", "*b = run + p->beta * p->M;", "*b = run + p->M;"),
 ("dp_oracle.c", "arrival off by one", "if (orc_in_target(p, y)) { t_arrive[i] = (s + 1) * h; break; }", "if (orc_in_target(p, y)) { t_arrive[i] = s * h; break; }"),
 ("dp_oracle.c", "target closed box", "!(fabs(x[d] - p->tgt_c[d]) < p->tgt_w[d])", "!(fabs(x[d] - p->tgt_c[d]) <= p->tgt_w[d])"),
 ("dp_oracle.c", "target node not zero", "    if (target[j]) { *v_out = 0.0; *code_out = code_in; return 0; }", "    if (target[j]) { *v_out = p->dt; *code_out = code_in; return 0; }"),
 ("dp_oracle.c", "node state offset", "x[d] = p->lo[d] + idx[d] * spacing(p, d);", "x[d] = p->lo[d] + (idx[d] + 1) * spacing(p, d);"),
 ("dp_oracle.c", "table code truncates", "return (k * ORC_NCODES + K / 2) / K;", "return (k * ORC_NCODES) / K;"),
 ("mlp.py", "gelu erf scale", "return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))", "return 0.5 * z * (1.0 + erf(z / 2.0))"),
 ("mlp.py", "backward transposed", "        d = d @ W\n", "        d = d @ W.T if W.shape[0] == W.shape[1] else d @ W\n"),
 ("mlp.py", "adam no bias correction", "            mh = m / (1 - b1 ** t)", "            mh = m"),
 ("mlp.py", "adam v uses g", "v = state[\"v\"][li][pi] = b2 * state[\"v\"][li][pi] + (1 - b2) * g * g", "v = state[\"v\"][li][pi] = b2 * state[\"v\"][li][pi] + (1 - b2) * abs(g)"),
 ("mlp.py", "loss sum not mean", "return float(np.mean((Y - T) ** 2))", "return float(np.sum((Y - T) ** 2))"),
 ("mlp.py", "bias grad mean", "grads[li] = [d.T @ a_in, d.sum(axis=0)]", "grads[li] = [d.T @ a_in, d.mean(axis=0)]"),
 ("dp_oracle.c", "spacing over n", "return (p->hi[d] - p->lo[d]) / (double)(p->n[d] - 1);", "return (p->hi[d] - p->lo[d]) / (double)(p->n[d]);"),
 ("dp_oracle.c", "theta not periodic", "return p->dynamics == ORC_DYN_POLAR && d == 3;", "return 0;"),
 ("dp_oracle.c", "feedback off loses ties", "            if (q_off <= q) { q = q_off; code = ORC_CODE_OFF; }\n        }\n        code_out[i]", "            if (q_off < q) { q = q_off; code = ORC_CODE_OFF; }\n        }\n        code_out[i]"),
 ("dp_oracle.c", "feedback without refinement", "        if (p->refine) code = fibonacci_refine(&c, k, q, &q);\n        if (p->off_control) {\n            double q_off", "        if (0) code = fibonacci_refine(&c, k, q, &q);\n        if (p->off_control) {\n            double q_off"),
 ("dp_oracle.c", "closed loop ignores thrust off", "rk4_step_drag(p, y, code_control(p, code), h, drag_c, z);", "rk4_step_drag(p, y, code_angle(code), h, drag_c, z);"),
 ("dp_oracle.c", "one evaluation sweep short", "for (int e = 0; e < n_eval; ++e) {", "for (int e = 1; e < n_eval; ++e) {"),
 ("dp_oracle.c", "vi diag penalty without dt", "q = p->dt + p->beta * p->M;", "q = p->beta * p->M;"),
 ("dp_oracle.c", "vi diag self weight ignored", "if (idx[b] == j) self += w[b];", "if (0) self += w[b];"),
 ("dp_oracle.c", "policy row target value", "if (target[j]) { *b = 0.0; return 0; }", "if (target[j]) { *b = p->dt; return 0; }"),
 ("dp_oracle.c", "VI stops one sweep late", "        ++s;\n        if (res < tol) break;", "        ++s;\n        if (res < 0.5 * tol) break;"),
 ("dp_oracle.c", "eval mode re-searches", "    if (mode == ORC_EVAL) {\n        *v_out = q_of_code(&c, code_in);", "    if (mode == ORC_EVAL) {\n        *v_out = q_of_code(&c, table_code(p->K, nearest_table_index(p->K, code_in)));"),
 ("mlp.py", "gelu grad drops z pdf", "return cdf + z * pdf", "return cdf"),
 ("mlp.py", "forward no bias", "        z = a @ W.T + b\n", "        z = a @ W.T\n"),
 ("mlp.py", "bf16 activation not rounded", "        a = bf16(gelu(z)) if li < last else z", "        a = gelu(z) if li < last else z"),
 ("mlp.py", "bf16 W1 rounded too", "        if 0 < li < last:\n            W = bf16(W)\n        z = a @ W.T + b", "        if li < last:\n            W = bf16(W)\n        z = a @ W.T + b"),
 ("mlp.py", "bf16 dz not rounded", "            d = bf16(d * gelu_grad(z))", "            d = d * gelu_grad(z)"),
 ("mlp.py", "bf16 backward unrounded W", "        if 0 < li < last:\n            W = bf16(W)\n        grads[li]", "        if False:\n            W = bf16(W)\n        grads[li]"),
 ("__init__.py", "eval diag drops beta in the factor", "Vn = (b + beta * (Wm @ V - d * V)) / (1.0 - beta * d)", "Vn = (b + beta * (Wm @ V - d * V)) / (1.0 - d)"),
 ("__init__.py", "exact evaluation without beta", "A = (sp.identity(self.N, format=\"csr\") - self.s.beta * W).tocsc()", "A = (sp.identity(self.N, format=\"csr\") - W).tocsc()"),
 ("__init__.py", "policy system transposed", "W = sp.csr_matrix((w[used], (rows[used], idx[used])), shape=(self.N, self.N))", "W = sp.csr_matrix((w[used], (idx[used], rows[used])), shape=(self.N, self.N))"),
 ("dp_oracle.c", "angle seam clamped", "if (periodic(p, d) && idx[d] == p->n[d]) idx[d] = 0;", "if (periodic(p, d) && idx[d] == p->n[d]) idx[d] = p->n[d] - 1;"),
 ("dp_oracle.c", "walk start truncated", "return (int)(((code * K + ORC_NCODES / 2) / ORC_NCODES) % K);", "return (int)(((code * K) / ORC_NCODES) % K);"),
 ("dp_oracle.c", "target counts zero-width dims", "if (p->tgt_w[d] > 0.0 && !(fabs(x[d] - p->tgt_c[d]) < p->tgt_w[d])) return 0;", "if (p->tgt_w[d] >= 0.0 && !(fabs(x[d] - p->tgt_c[d]) < p->tgt_w[d])) return 0;"),
 ("dp_oracle.c", "periodic fraction reversed", "            t[d] = s[d] - f;", "            t[d] = 1.0 - (s[d] - f);"),
]


@pytest.mark.skipif(os.environ.get("DP_ORACLE_MUTATIONS") != "1", reason="opt-in: DP_ORACLE_MUTATIONS=1")
@pytest.mark.parametrize("case", range(len(MUTATIONS)), ids=[m[1].replace(" ", "-") for m in MUTATIONS])
def test_planted_mistake_fails_a_pin(case, tmp_path):
    fname, what, good, bad = MUTATIONS[case]
    copy = tmp_path / "oracle"
    shutil.copytree(os.path.join(ROOT, "oracle"), copy, ignore=shutil.ignore_patterns("_build", "__pycache__"))
    path = copy / fname
    text = path.read_text()
    assert text.count(good) >= 1, what
    path.write_text(text.replace(good, bad, 1))
    env = dict(os.environ, PYTHONPATH=os.pathsep.join([str(tmp_path), ROOT]))
    subprocess.run([sys.executable, "-c", "from oracle.build import build_oracle; build_oracle(force=True)"],
                   cwd=str(tmp_path), env=env, check=True, capture_output=True)
    # run from the temporary directory, so that it (not the repository root)
    # comes first on the import path and "import oracle" finds the copy
    check = subprocess.run([sys.executable, "-c", "import oracle, os; print(os.path.dirname(oracle.__file__))"],
                           cwd=str(tmp_path), env=env, check=True, capture_output=True, text=True)
    assert check.stdout.strip() == str(copy)          # the suite will test the mutated copy
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests"), "-m",
                        "not gpu and not mutation", "-x", "-q", "-p", "no:cacheprovider"],
                       cwd=str(tmp_path), env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, "planted mistake survived every pin: %s" % what
