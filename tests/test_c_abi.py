"""The C ABI used from C: tests/c_abi_solve.c includes only include/adr.h and
links only libadr_gb300.so.  It compiles on any host; on a GPU its result
equals the Python binding's bit for bit and matches the FP64 oracle."""
import os
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
import workloads as wl
from oracle import schemes

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "c_abi_solve.c")


def problem(nsteps=20):
    # the problem hard-wired in c_abi_solve.c
    return wl.Problem(d=2, n=(96, 64), lo=(0.0, 0.0), hi=(100.0, 100.0), diff=(1.0, 20.0),
                      adv=((0.5, 0.5), (0.5, 0.5)), model=wl.FHN, params=(0.05, 2.0, -0.03),
                      tau=1e-2, nsteps=nsteps, precision=wl.BF16X3, seed=7, name="c_abi_fhn")


def compile_program(outdir):
    from paper_2307_10684_gb300 import build
    build.build()
    libdir = os.path.dirname(build.LIB)
    exe = os.path.join(outdir, "c_abi_solve")
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), SRC,
                    "-o", exe, "-L", libdir, "-ladr_gb300", "-Wl,-rpath," + libdir],
                   check=True, capture_output=True, text=True)
    return exe


def test_c_program_compiles_against_the_header():
    with tempfile.TemporaryDirectory() as d:
        assert os.path.exists(compile_program(d))


@pytest.mark.gpu
def test_c_program_matches_binding_and_oracle():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2307_10684_gb300 as adr
    p = problem()
    u0, v0 = wl.initial_data(p)
    u0 = np.asarray(wl.round_to(u0, wl.FP32), dtype=np.float32)
    v0 = np.asarray(wl.round_to(v0, wl.FP32), dtype=np.float32)
    with tempfile.TemporaryDirectory() as d:
        exe = compile_program(d)
        fin, fout = os.path.join(d, "in.f32"), os.path.join(d, "out.f32")
        np.concatenate([u0.ravel(), v0.ravel()]).tofile(fin)
        r = subprocess.run([exe, str(p.nsteps), fin, fout], capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
        out = np.fromfile(fout, dtype=np.float32)
    N = u0.size
    uc, vc = out[:N].reshape(u0.shape), out[N:].reshape(v0.shape)
    u = torch.tensor(u0, device="cuda")
    v = torch.tensor(v0, device="cuda")
    with adr.Plan(p) as plan:
        plan.step(u, v, p.nsteps)
    torch.cuda.synchronize()
    assert np.array_equal(u.cpu().numpy(), uc) and np.array_equal(v.cpu().numpy(), vc)
    Ur, Vr = schemes.etd2rkds_solve(schemes.make_plan(p), u0.astype(np.float64),
                                    v0.astype(np.float64), p.nsteps)
    assert oracle.max_rel_err(uc.astype(np.float64), vc.astype(np.float64), Ur, Vr) <= 1e-5
