"""The oracle's pins catch planted mistakes (CPU only, gcc).

Every mutant of oracle/gp_oracle.c listed in tests/oracle_mutants.py is
compiled into a library of its own and the pins are run against it in a
child process; each mutant must fail at least one pin.  The unchanged
source, compiled and loaded the same way, must pass every pin, so a failure
is the mutant's doing and not the harness's.
"""
import json
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

from oracle import oracle as O
from tests.oracle_mutants import MUTANTS, mutate

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def compile_and_run(src: str, work: str, tag: str, run_all: bool = False) -> dict:
    c_path = os.path.join(work, f"{tag}.c")
    so_path = os.path.join(work, f"lib{tag}.so")
    with open(c_path, "w") as f:
        f.write(src)
    subprocess.run(["gcc", *O.CFLAGS, "-o", so_path, c_path, "-lm"], check=True,
                   capture_output=True, timeout=120)
    cmd = [sys.executable, "-m", "tests.oracle_mutants", so_path] + (["--all"] if run_all else [])
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    if r.returncode != 0 or not lines:
        return {"crashed": r.returncode, "stderr": r.stderr[-400:]}
    return json.loads(lines[-1])


@pytest.fixture(scope="module")
def source():
    with open(O._SRC) as f:
        return f.read()


def test_mutant_texts_are_unique_edits(source):
    names = [m[0] for m in MUTANTS]
    assert len(set(names)) == len(names)
    for name, find, repl, occ in MUTANTS:
        assert mutate(source, find, repl, occ) != source, name


def test_every_planted_mistake_fails_a_pin(source, tmp_path):
    work = str(tmp_path)
    jobs = [("control", source, True)] + [
        (f"m{k:02d}", mutate(source, find, repl, occ), False)
        for k, (name, find, repl, occ) in enumerate(MUTANTS)]
    with ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
        res = list(ex.map(lambda j: compile_and_run(j[1], work, j[0], j[2]), jobs))
    control, muts = res[0], res[1:]
    assert "crashed" not in control, control
    assert control["failed"] == [], control["failed"]
    survivors = [MUTANTS[k][0] for k, r in enumerate(muts) if "crashed" in r or not r["failed"]]
    assert survivors == [], survivors
