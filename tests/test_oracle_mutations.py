"""Planted mistakes in the oracle must fail its pins.

Each entry below copies oracle.c with one plausible mistake (a dropped term, a wrong sign,
factor or index, a missing rule of the hit test), compiles the copy on the CPU and runs the
pin files that should catch it against that library (ORACLE_LIB).  Every mutant has to make
at least one pin fail: a pin set that lets a mistake through is not pinning that part.  The
unmutated oracle passes the same files in the rest of the suite (no GPU)."""
import concurrent.futures
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")

# (mistake, text in oracle.c, replacement, pin files that must catch it)
MUTANTS = [
    # hemisphere transport (Eq. L_I, Sec. 5.2)
    ("compositing drops the (1 - alpha) of nearer hits",
     "            s->hit_a[e] = per[r].h[q].alpha * T;\n            T *= (1.0 - per[r].h[q].alpha);",
     "            s->hit_a[e] = per[r].h[q].alpha * T;\n            T *= 1.0;", ["transport"]),
    ("shadow rays ignore occluders",
     "for (int q = 0; q < hv->cnt; ++q) T *= (1.0 - hv->h[q].alpha);",
     "for (int q = 0; q < hv->cnt; ++q) T *= 1.0;", ["transport"]),
    ("direct term evaluates the lobe without the reflection R_i",
     "            reflect(s->nrm + i * 3, w, rw);\n            or_sh_eval(L, rw, Y);\n            for (int kk = 0; kk < nc; ++kk)\n"
     "                for (int ch = 0; ch < 3; ++ch)\n                    s->Dgeo",
     "            memcpy(rw, w, sizeof rw);\n            or_sh_eval(L, rw, Y);\n            for (int kk = 0; kk < nc; ++kk)\n"
     "                for (int ch = 0; ch < 3; ++ch)\n                    s->Dgeo", ["transport"]),
    ("the gather reads the source's radiance along d instead of -d",
     "            for (int q = 0; q < 3; ++q) md[q] = -d[q];\n            reflect(s->nrm + i * 3, d, rd);\n"
     "            or_sh_eval(L, md, Yo);\n            or_sh_eval(L, rd, Yi);\n            long ray = (long)i * nd + r;\n"
     "            for (int c = 0; c < C; ++c) x[c] = 0.0;",
     "            for (int q = 0; q < 3; ++q) md[q] = d[q];\n            reflect(s->nrm + i * 3, d, rd);\n"
     "            or_sh_eval(L, md, Yo);\n            or_sh_eval(L, rd, Yi);\n            long ray = (long)i * nd + r;\n"
     "            for (int c = 0; c < C; ++c) x[c] = 0.0;", ["transport"]),
    ("no eps_plane rule for planes through the ray origin",
     "    if (fabs(h) <= s->eps_plane) return;", "    (void)h;", ["transport"]),
    ("no tie runs for near-equal depths",
     "            if (e > k) qsort(out->h + k, (size_t)(e - k + 1), sizeof(or_hit), cmp_hit_j);",
     "            (void)cmp_hit_j;", ["transport"]),
    ("Gaussian exp(-r^2) instead of exp(-r^2 / 2)",
     "        G = exp(-0.5 * r2);\n    }\n    or_hit x", "        G = exp(-r2);\n    }\n    or_hit x",
     ["transport", "pairs"]),
    ("3-sigma cutoff at 2 sigma",
     "        if (r2 > 9.0) return;\n        G = exp(-0.5 * r2);", "        if (r2 > 4.0) return;\n        G = exp(-0.5 * r2);",
     ["transport", "pairs", "gfsgs", "lights"]),
    ("disc model of radius 2",
     "        if (r2 > 1.0) return;\n        G = 1.0;", "        if (r2 > 4.0) return;\n        G = 1.0;",
     ["transport", "pairs"]),
    ("BVH slab test keeps the far slab distance as the entry",
     "        if (ta > t0) t0 = ta;", "        if (ta > t0) t0 = tb;", ["transport", "pairs"]),
    ("Malley mapping with radius sqrt(1 - u)",
     "    double rr = sqrt(u1), ph = 2.0 * OR_PI * u2;", "    double rr = sqrt(1.0 - u1), ph = 2.0 * OR_PI * u2;",
     ["math", "transport"]),
    ("strata indices swapped",
     "    int a = r / nb, b = r % nb;", "    int a = r % na, b = r / na;", ["math"]),
    ("rays in the world frame instead of the receiver's",
     "    for (int q = 0; q < 3; ++q) d[q] = c[0] * s->tu[i * 3 + q] + c[1] * s->tv[i * 3 + q] + c[2] * s->nrm[i * 3 + q];",
     "    for (int q = 0; q < 3; ++q) d[q] = c[q];", ["transport", "math"]),
    ("lights behind the receiver contribute",
     "    if (!(cs > 0.0)) return 0.0; /* only the front hemisphere Omega receives */", "    /* none */",
     ["transport", "lights"]),
    ("point light falls off as 1/r instead of 1/r^2",
     "    return s->ldir ? cs : cs / (len * len);", "    return s->ldir ? cs : cs / len;", ["transport"]),
    ("emission added to the first light's columns only",
     "                for (int c = 0; c < C; ++c) S[((size_t)i * nc + kk) * C + c] += E[((size_t)i * nc + kk) * 3 + c % 3];",
     "                for (int c = 0; c < 3; ++c) S[((size_t)i * nc + kk) * C + c] += E[((size_t)i * nc + kk) * 3 + c % 3];",
     ["transport", "lights", "pairs"]),
    ("dL/dE summed over the first light's columns only",
     "                    for (int lt = 0; lt < C / 3; ++lt) acc += u[((size_t)i * nc + kk) * C + lt * 3 + ch];",
     "                    for (int lt = 0; lt < 1; ++lt) acc += u[((size_t)i * nc + kk) * C + lt * 3 + ch];",
     ["transport", "lights", "pairs"]),
    ("albedo gradient without the direct term's share",
     "                double acc = u[idx] * s->Dgeo[idx];", "                double acc = 0.0 * s->Dgeo[idx];", ["transport"]),
    ("albedo gradient without the blend weight k",
     "dad[i * 3 + ch] = 4.0 * s->k[i] * alpha_c(s, i) * P[", "dad[i * 3 + ch] = 4.0 * alpha_c(s, i) * P[",
     ["transport"]),
    ("compositing backward without the later hits' share R",
     "                    double dalpha = Th[h] * (gh[h] - R);", "                    double dalpha = Th[h] * gh[h];",
     ["transport"]),
    ("directional light's shadow ray stops at the direction vector's length",
     "    *r = s->ldir ? INFINITY : len;", "    *r = len;", ["lights"]),
    ("albedo gradient pairs v^(a) with Q^(a) instead of Q^(n-1-a)",
     "acc += v[(size_t)a * M + idx] * Q[(size_t)(nb - 1 - a) * M + idx];",
     "acc += v[(size_t)a * M + idx] * Q[(size_t)a * M + idx];", ["transport"]),
    # BRDF, SH, ray keys (Eq. brdf, App. A, App. B)
    ("diffuse coefficient k a^d instead of 4 k a^d",
     "4.0 * k * ad[ch] + (1.0 - k) * as[ch]", "k * ad[ch] + (1.0 - k) * as[ch]", ["math"]),
    ("Phong factor of odd bands with a shifted denominator",
     "for (int q = 2; q <= l + 1; q += 2) den *= (s + q);", "for (int q = 2; q <= l + 1; q += 2) den *= (s + q + 1);",
     ["math"]),
    ("SH without the Condon-Shortley phase",
     "for (int q = 1; q <= m; ++q) pmm *= -(2.0 * q - 1.0); /* (-1)^m",
     "for (int q = 1; q <= m; ++q) pmm *= (2.0 * q - 1.0); /* (-1)^m", ["math"]),
    ("SplitMix64 with a wrong multiplier",
     "z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;", "z = (z ^ (z >> 27)) * 0x94D049BB133111EDULL;", ["math"]),
    ("Phong factor of even bands with a shifted numerator",
     "        for (int q = 0; q >= -(l - 2); q -= 2) num *= (s + q);",
     "        for (int q = 0; q >= -(l - 2); q -= 2) num *= (s + q + 1);", ["math"]),
    ("specular coefficients weighted by k instead of 1 - k",
     "(1.0 - k) * as[ch] * or_phong_rho(l, shin)", "k * as[ch] * or_phong_rho(l, shin)", ["math", "transport"]),
    ("jitter on [0, 1/2) (one bit short)",
     "    return (double)(or_splitmix64(key) >> 40) * (1.0 / 16777216.0);",
     "    return (double)(or_splitmix64(key) >> 41) * (1.0 / 16777216.0);", ["math"]),
    ("eps_plane a hundred times too wide",
     "    s->eps_plane = 1e-5 * sqrt(diag);", "    s->eps_plane = 1e-3 * sqrt(diag);", ["transport", "pairs"]),
    ("tie runs a thousand times too wide",
     "            while (e + 1 < out->cnt && out->h[e + 1].t - out->h[e].t <= 1e-6 * fmax(1.0, out->h[e].t)) ++e;",
     "            while (e + 1 < out->cnt && out->h[e + 1].t - out->h[e].t <= 1e-3 * fmax(1.0, out->h[e].t)) ++e;",
     ["transport"]),
    ("hit opacity ignores the surfel's o",
     "    or_hit x = {t, alpha_of(s, s->o[j], G), G, j};", "    or_hit x = {t, alpha_of(s, 1.0, G), G, j};",
     ["transport", "pairs"]),
    ("directional light without the receiver's cosine",
     "    return s->ldir ? cs : cs / (len * len);", "    return s->ldir ? 1.0 : cs / (len * len);", ["lights"]),
    ("opacity receiver term with alpha instead of d alpha / d o",
     "            dop[i] = dalpha_c(s, i) * acc;", "            dop[i] = alpha_c(s, i) * acc;", ["gfsgs", "transport"]),
    ("shadow-ray opacity backward with the wrong sign",
     "                    dop[s->sh_j[e]] += -qv * others * dalpha_do(s, s->o[s->sh_j[e]], s->sh_G[e]);",
     "                    dop[s->sh_j[e]] += qv * others * dalpha_do(s, s->o[s->sh_j[e]], s->sh_G[e]);", ["transport"]),
    # center-to-center transport (Sec. 8, App. E)
    ("pair transport without the source's cosine",
     "double geo = fabs(dot3(s->nrm + i * 3, d)) * fabs(dot3(s->nrm + j * 3, d)) / r2;",
     "double geo = fabs(dot3(s->nrm + i * 3, d)) / r2;", ["pairs"]),
    ("pair segments ignore occluders",
     "for (int q = 0; q < occ[e].cnt; ++q) T *= 1.0 - occ[e].h[q].alpha;",
     "for (int q = 0; q < occ[e].cnt; ++q) T *= 1.0;", ["pairs"]),
    ("Gaussian alpha integral without the 3-sigma truncation",
     "    return 2.0 * OR_PI * s->su[j] * s->sv[j] * (1.0 - exp(-4.5));", "    return 2.0 * OR_PI * s->su[j] * s->sv[j];",
     ["pairs"]),
    ("pair front test without eps_plane",
     "            if (dot3(s->nrm + i * 3, d) > s->eps_plane) cnt[i]++;",
     "            if (dot3(s->nrm + i * 3, d) > -1.0) cnt[i]++;", ["pairs"]),
    ("occluders within eps_plane of the source's plane kept",
     "        if (fabs(dot3(nk, e)) <= s->eps_plane) continue;", "        (void)e;", ["pairs"]),
    ("pair opacity gradient without lambda",
     "                dop[j] += g * s->lam[j] * dA * T * geo;", "                dop[j] += g * dA * T * geo;", ["pairs"]),
    ("lambda gradient without the alpha integral",
     "if (dlam) dlam[j] += g * A * T * geo;", "if (dlam) dlam[j] += g * T * geo;", ["pairs"]),
    ("GFSGS opacity derivative without the exponent 3.4",
     "        return exp(-p) * 3.4 * p / o;", "        return exp(-p) * p / o;", ["gfsgs"]),
    ("lambda left out of the pair transport",
     "            s->pair_V[e] = s->lam[j] * or_alpha_area(s, j) * T * geo;",
     "            s->pair_V[e] = or_alpha_area(s, j) * T * geo;", ["pairs"]),
    ("GFSGS receiver factor o instead of alpha_i(p_i)",
     "static double alpha_c(const or_scene *s, int i) { return alpha_of(s, s->o[i], 1.0); }",
     "static double alpha_c(const or_scene *s, int i) { return s->o[i]; }", ["gfsgs"]),
    ("GFSGS exponent 3 instead of 3.4",
     "        return -expm1(-0.03279 * pow(x, 3.4));", "        return -expm1(-0.03279 * pow(x, 3.0));", ["gfsgs"]),
    ("Ein series without its alternating sign",
     "            term *= -x / k;", "            term *= x / k;", ["gfsgs"]),
    # geometry gradients (Eqs. dl-dgeo-0/1)
    ("hemisphere ray's t^u share of the direction gradient not passed to the frame",
     "                        gF[i * 9 + a] += c3[0] * gd[a];", "                        gF[i * 9 + a] += 0.0 * gd[a];",
     ["geometry"]),
    ("hemisphere ray's normal share with t^v's coefficient",
     "                        gF[i * 9 + 6 + a] += c3[2] * gd[a];", "                        gF[i * 9 + 6 + a] += c3[1] * gd[a];",
     ["geometry"]),
    ("lobe reflection's normal derivative without its factor 2",
     "    for (int a = 0; a < 3; ++a) gn[a] += 2.0 * (ng * w[a] + nw * gR[a]);",
     "    for (int a = 0; a < 3; ++a) gn[a] += (ng * w[a] + nw * gR[a]);", ["geometry"]),
    ("crossing point's normal derivative with the wrong sign",
     "const double fn = -dot3(gx, d) / dot3(nk, d);", "const double fn = dot3(gx, d) / dot3(nk, d);", ["geometry"]),
    ("occluder crossing moves the ray origin with the wrong sign",
     "        gpo[a] += coef * pw[a];\n        gd[a] += coef * t * pw[a];",
     "        gpo[a] -= coef * pw[a];\n        gd[a] += coef * t * pw[a];", ["geometry"]),
    ("crossing's direction derivative without the depth t",
     "        gd[a] += coef * t * pw[a];\n        if (dp)", "        gd[a] += coef * pw[a];\n        if (dp)", ["geometry"]),
    ("occluder's t^v derivative with u for v",
     "            gF[k * 9 + 3 + a] += coef * 2.0 * v * xm[a] / s->sv[k];",
     "            gF[k * 9 + 3 + a] += coef * 2.0 * u * xm[a] / s->sv[k];", ["geometry"]),
    ("decay term's distance derivative -geo/r instead of -2 geo/r",
     "const double gr = ge * lam * A * T * (-2.0 * geo / r);", "const double gr = ge * lam * A * T * (-geo / r);",
     ["geometry"]),
    ("occluder scale derivative with half its factor",
     "        ds[k * 2] += coef * (-2.0 * u * u / s->su[k]);", "        ds[k * 2] += coef * (-u * u / s->su[k]);",
     ["geometry"]),
    ("source scale gradient dropped",
     "            ds[j * 2] += ge * lam * T * geo * A / s->su[j];", "            ds[j * 2] += 0.0 * ge;", ["geometry"]),
    # Monte-Carlo solver, progressive refinement (Sec. 7, Alg. 1)
    ("one-point estimate without the 1/p weight",
     "                                s->pair_V[e] * sv / p;", "                                s->pair_V[e] * sv;",
     ["mc"]),
    ("reservoir keeps candidates with twice their probability",
     "if (mc_u(seed, (uint64_t)t, (uint64_t)q, 1000 + (uint64_t)k) * W < w[k]) pick = k;",
     "if (mc_u(seed, (uint64_t)t, (uint64_t)q, 1000 + (uint64_t)k) * W < 2.0 * w[k]) pick = k;", ["mc"]),
    ("grouped proposal's probability without the group's share",
     "        if (pick >= 0) *p = wg[gsel] / totg * wk[pick] / totk;", "        if (pick >= 0) *p = wk[pick] / totk;", ["mc"]),
    ("visit count advances by two",
     "            D[a] += 1.0;", "            D[a] += 2.0;", ["mc"]),
    ("receiver selection by the second moment instead of the variance",
     "                    v += SB2[i * R + k] / D[i] - m * m;", "                    v += SB2[i * R + k] / D[i];", ["mc"]),
    ("TD(0) mean not divided by the visits",
     "                for (size_t k = 0; k < R; ++k) Bhat[i * R + k] = SB[i * R + k] / D[i];",
     "                for (size_t k = 0; k < R; ++k) Bhat[i * R + k] = SB[i * R + k];", ["mc"]),
    ("proposal without its floor",
     "    return 1e-9 * (1.0 + acc / (double)s->n);", "    return 0.0 * acc;", ["mc"]),
    ("shooting takes the dimmest unshot surfel",
     "            if (l > bl) {\n                bl = l;\n                best = i;",
     "            if (l > 0.0 && (best < 0 || l < bl)) {\n                bl = l;\n                best = i;", ["mc"]),
    ("shooting leaves the shot radiance unshot",
     "        memset(dB + (size_t)best * R, 0, sizeof(double) * R);", "        (void)best;", ["mc"]),
    # image formation (Eq. L_I for a camera)
    ("pixel rays through pixel corners instead of centres",
     "    const double sx = (2.0 * (x + 0.5) / W - 1.0) * th * (double)W / (double)H;",
     "    const double sx = (2.0 * x / W - 1.0) * th * (double)W / (double)H;", ["render"]),
    ("image rows not flipped (y up)",
     "    const double sy = (1.0 - 2.0 * (y + 0.5) / H) * th;", "    const double sy = (2.0 * (y + 0.5) / H - 1.0) * th;",
     ["render"]),
    ("camera up taken as given instead of right x forward",
     "    cross3(r, fn, u);\n    const double th", "    for (int a = 0; a < 3; ++a) u[a] = u0[a];\n    const double th",
     ["render"]),
    ("image transpose drops the radiance direction's SH",
     "                            dB[((size_t)j * nc + k) * C + c] += g * Yo[k];",
     "                            dB[((size_t)j * nc + k) * C + c] += g;", ["render"]),
    ("camera rays ignore the transmittance of nearer surfels",
     "                T *= 1.0 - hv.h[h].alpha;\n                const int j = hv.h[h].j;",
     "                T *= 1.0;\n                const int j = hv.h[h].j;", ["render"]),
]


def _run_mutant(tmp, index, old, new, files):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutant {index}: the text to replace must occur exactly once"
    c_path = os.path.join(tmp, f"mutant{index}.c")
    so_path = os.path.join(tmp, f"mutant{index}.so")
    with open(c_path, "w") as f:
        f.write(src.replace(old, new, 1))
    subprocess.run(["gcc", "-O1", "-std=c11", "-fopenmp", "-shared", "-fPIC", "-o", so_path, c_path, "-lm"],
                   check=True, capture_output=True)
    env = dict(os.environ, ORACLE_LIB=so_path, OMP_NUM_THREADS="2")
    paths = [os.path.join(ROOT, "tests", f"test_oracle_{f}.py") for f in files]
    proc = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", *paths],
                          cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return proc.returncode, proc.stdout[-2000:]


def test_every_planted_mistake_fails_a_pin(tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    workers = max(1, min(4, (os.cpu_count() or 2) // 2))
    with concurrent.futures.ThreadPoolExecutor(workers) as ex:
        futs = [ex.submit(_run_mutant, str(tmp_path), q, old, new, files)
                for q, (_, old, new, files) in enumerate(MUTANTS)]
        results = [f.result() for f in futs]
    survived = []
    for (name, _, _, files), (rc, out) in zip(MUTANTS, results):
        # 1: a pin failed; a negative code: the mutant crashed the run.  0 means it went
        # unnoticed; 2-5 mean pytest itself could not run the files.
        if rc == 0 or rc in (2, 3, 4, 5):
            survived.append(f"{name} (files {files}, exit {rc}):\n{out}")
    assert not survived, "planted mistakes the pins did not catch:\n" + "\n".join(survived)
