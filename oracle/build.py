"""Build the oracle's C library (test infrastructure): gcc -O2 -ffp-contract=off -shared."""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))


def build_oracle(force: bool = False) -> str:
    src = os.path.join(HERE, "mgm_oracle.c")
    out = os.path.join(HERE, "liboracle.so")
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(src):
        return out
    tmp = out + f".tmp{os.getpid()}"
    subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                    "-Wall", "-Wno-unused-function", "-o", tmp, src, "-lm"], check=True)
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build_oracle(force=True))
