"""Writes tests/golden/pml_tables_oracle.txt: the FP64 oracle's errors for the paper's ADE-PML study (Sec. 4.1,
Tables PML_error_L_t020, err_PML_R and err_PML_kmax) on 512^2 intervals, and for the rows of Table 2d_error
after the wave has left the domain (t >= 0.1 s) on 64^2 .. 256^2 intervals with the layer of the 512^2 runs.

The Gaussian pulse of Sec. 4.1 runs on [-5, 5]^2 padded by L points on every side, with the absorbing layer in the
padding: thickness L points, reflection coefficient R, cut-off k_max, and f_P = c_P / L with L in points as
printed (1 Hz for the paper's L = 50), alpha_max = pi f_P.
Every 200 steps (dt = 1e-4, up to t = 0.2 s), v3 inside [-5, 5]^2 is compared with the free-space solution of the
same time stepping (oracle/exact.py).  Per configuration and time the file holds the relative l2 error, the
paper's eps_2 read literally (l2 norm of the error / max |v3_ref| at that time), and eps_2 with the area element
and one amplitude for the whole run, h ||e||_2 / A with A the largest |v3_ref| over t <= 0.2 s (the reading whose
values agree with the paper's printed ones).

Only oracle/ and synth/ are called.  Run from the repository root:

    python tests/golden/make_pml_tables.py

The configurations run in parallel processes, one thread each, about 5 minutes each on the 613^2 grid.
"""
import dataclasses
import multiprocessing as mp
import os
import sys

# (N, L, R, k_max): on 512^2 the thickness study at R = 1e-6, k_max = 1, the R study at L = 50 and the k_max
# study at L = 50; on 64^2 .. 256^2 the convergence rows with L = 50 and R = 1e-6 or 1e-9
CONFIGS = [(512, 10, 1e-6, 1.0), (512, 20, 1e-6, 1.0), (512, 50, 1e-6, 1.0),
           (512, 50, 1e-1, 1.0), (512, 50, 1e-3, 1.0), (512, 50, 1e-9, 1.0),
           (512, 50, 1e-6, 0.5), (512, 50, 1e-6, 6.0)] + \
          [(n, 50, R, 1.0) for n in (64, 128, 256) for R in (1e-6, 1e-9)]
TIMES = tuple(range(200, 2001, 200))  # steps of 1e-4 s: 0.02 .. 0.20 s


def run(cfg):
    os.environ["OPENBLAS_NUM_THREADS"] = "1"
    root = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    sys.path.insert(0, root)
    import numpy as np

    from oracle.exact import pulse_on_grid
    from oracle.wave import Simulation
    from synth import gaussian_pulse_2d

    N, L, R, kmax = cfg
    w, s0 = gaussian_pulse_2d(N, p=2, n_nb=20, dt=1e-4, steps=TIMES[-1], pad=L)
    w = dataclasses.replace(w, pml_width=L, pml_R=R, pml_kmax=kmax, f0=50.0 / L)
    sim = Simulation(w, state={"sigma": s0, "v1": 0 * s0, "v3": 0 * s0})
    # the run's largest |v3_ref|: v3 peaks early, while the pulse separates from the centre
    A = max(float(np.abs(pulse_on_grid(N, k, 1e-4)[1]).max()) for k in list(range(50, 401, 25)) + list(TIMES))
    out, done = [], 0
    for steps in TIMES:
        sim.step(steps - done, record=False)
        done = steps
        ref = pulse_on_grid(N, steps, 1e-4)[1]
        e = sim.state["v3"][L:L + N + 1, L:L + N + 1] - ref
        en = float(np.linalg.norm(e))
        out.append((steps, en / float(np.linalg.norm(ref)), en / float(np.abs(ref).max()), w.h[0] * en / A))
    return cfg, out


def main():
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(len(CONFIGS), os.cpu_count() or 1)) as pool:  # the 512^2 runs first: they take longest
        results = pool.map(run, CONFIGS)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "pml_tables_oracle.txt")
    with open(path, "w") as f:
        f.write("# FP64 oracle, Gaussian pulse of Sec. 4.1 on N^2 intervals padded by L points with the layer in the\n")
        f.write("# padding (Tables PML_error_L_t020, err_PML_R, err_PML_kmax, 2d_error); written by\n")
        f.write("# tests/golden/make_pml_tables.py.\n")
        f.write("# columns: N  L  R  k_max  steps  rel_l2(v3)  ||e||_2 / max|v3_ref(t)|  h ||e||_2 / A\n")
        for (N, L, R, kmax), rows in results:
            for steps, rel, eps2, eps2a in rows:
                f.write(f"{N} {L} {R:.0e} {kmax} {steps} {rel:.6e} {eps2:.6e} {eps2a:.6e}\n")
    print("wrote", path)


if __name__ == "__main__":
    main()
