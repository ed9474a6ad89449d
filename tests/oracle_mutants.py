"""Mutation check of the oracle's pins (test infrastructure; run by hand).

Each entry of ``oracle_mutants.json`` plants one plausible mistake in
``oracle/pic_oracle.c``: a dropped factor, a flipped sign, a wrong time level,
a transposed stagger, an upwind difference taken on the wrong side, a stencil
point off by one, a mis-keyed random stream.  The script copies the oracle
and the CPU oracle tests into a temporary directory, applies one mistake at a
time, rebuilds the oracle there and runs the pins.  A mistake that passes every
pin marks a part of the oracle that nothing independent fixes.  The repository's
own oracle is never modified.

    python tests/oracle_mutants.py [name ...]

Prints one line per mistake (KILLED or SURVIVED) and exits 1 if any survived.
An entry with an ``unpinned_on_cpu`` reason is a change that no CPU pin can
see by design (a convention only the GPU parity tests hold both sides to);
it is reported as such and does not fail the check, and must not be caught
(if a pin catches it, the reason is stale).  About five seconds per mistake
on one core.
"""
from __future__ import annotations

import json
import os
import shutil
import subprocess
import sys
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def stage(dst: str) -> None:
    ign = shutil.ignore_patterns("_build", "__pycache__")
    shutil.copytree(os.path.join(ROOT, "oracle"), os.path.join(dst, "oracle"), ignore=ign)
    os.makedirs(os.path.join(dst, "tests"))
    for f in os.listdir(HERE):
        if f.startswith("test_oracle_") or f == "conftest.py":
            shutil.copy(os.path.join(HERE, f), os.path.join(dst, "tests", f))
    shutil.copytree(os.path.join(HERE, "golden"), os.path.join(dst, "tests", "golden"))
    # the seeded input generators (no arithmetic of the method) that some pins use
    pkg = os.path.join(dst, "paper_2602_15939_gb300")
    os.makedirs(pkg)
    for f in ("__init__.py", "workloads.py"):
        shutil.copy(os.path.join(ROOT, "paper_2602_15939_gb300", f), os.path.join(pkg, f))


def plant(src: str, old: str, new: str, count: int) -> str:
    n = src.count(old)
    if n != count:
        raise ValueError(f"pattern found {n} times, expected {count}")
    return src.replace(old, new)


def run(dst: str, mutant: dict, clean: str) -> tuple[bool, str]:
    with open(os.path.join(dst, "oracle", "pic_oracle.c"), "w") as f:
        f.write(plant(clean, mutant["old"], mutant["new"], mutant.get("count", 1)))
    shutil.rmtree(os.path.join(dst, "oracle", "_build"), ignore_errors=True)
    r = subprocess.run([sys.executable, "-m", "pytest", "tests", "-x", "-q", "-m", "not gpu", "-p", "no:cacheprovider"],
                       cwd=dst, capture_output=True, text=True, timeout=900)
    lines = r.stdout.strip().splitlines()
    return r.returncode != 0, lines[-1] if lines else r.stderr[-200:]


def main(argv: list[str]) -> int:
    with open(os.path.join(HERE, "oracle_mutants.json")) as f:
        mutants = json.load(f)
    if argv:
        mutants = [m for m in mutants if m["name"] in argv]
    with open(os.path.join(ROOT, "oracle", "pic_oracle.c")) as f:
        clean = f.read()
    survived = stale = 0
    with tempfile.TemporaryDirectory(prefix="oracle_mutants_") as dst:
        stage(dst)
        failed, tail = run(dst, {"old": "", "new": "", "count": clean.count("")}, clean)
        if failed:  # the unmodified copy must pass, or every mistake would look caught
            print(f"the unmodified oracle fails its pins: {tail}")
            return 2
        for m in mutants:
            killed, tail = run(dst, m, clean)
            if "unpinned_on_cpu" in m:
                stale += killed
                verdict = "KILLED (reason stale)" if killed else "not pinned on CPU"
            else:
                survived += not killed
                verdict = "KILLED" if killed else "SURVIVED"
            print(f"{m['name']:32s} {verdict}  {tail}", flush=True)
    known = sum("unpinned_on_cpu" in m for m in mutants)
    print(f"{len(mutants) - known - survived} of {len(mutants) - known} mistakes caught by the pins; "
          f"{known} listed as not pinned on the CPU")
    return 1 if survived or stale else 0


if __name__ == "__main__":
    sys.exit(main(sys.argv[1:]))
