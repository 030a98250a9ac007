"""Race and memory checks of the host code, on the CPU: the multi-threaded
graph builder and the graph-file code under ThreadSanitizer and under
AddressSanitizer + UBSan, and the oracle under AddressSanitizer + UBSan
(drivers: host_sanitize_driver.cpp, oracle_sanitize_driver.c).  The GPU code
is not covered here."""
import os
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_1603_09320_gb300", "csrc")
INCLUDE = os.path.join(ROOT, "include")
ORACLE = os.path.join(ROOT, "oracle")


def _supports(compiler, flag, tmp_path):
    src = tmp_path / "probe.c"
    src.write_text("int main(void) { return 0; }\n")
    r = subprocess.run([compiler, flag, str(src), "-o", str(tmp_path / "probe")], capture_output=True)
    return r.returncode == 0


def _run(cmd, env_extra, timeout=300):
    env = dict(os.environ, **env_extra)
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=timeout, env=env)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "ThreadSanitizer" not in r.stderr and "runtime error" not in r.stderr, r.stderr[-4000:]
    assert "Sanitizer" not in r.stderr, r.stderr[-4000:]
    return r.stdout


def _build_host(tmp_path, san):
    exe = tmp_path / f"host_{san.split(',')[0]}"
    cmd = ["g++", "-std=c++17", f"-fsanitize={san}", "-fno-omit-frame-pointer", "-g", "-O1", "-I", INCLUDE,
           os.path.join(CSRC, "builder.cpp"), os.path.join(CSRC, "blob.cpp"),
           os.path.join(HERE, "host_sanitize_driver.cpp"), "-o", str(exe), "-pthread"]
    if "undefined" in san:
        cmd.insert(3, "-fno-sanitize-recover=undefined")
    subprocess.run(cmd, check=True, capture_output=True, timeout=300)
    return exe


def test_builder_under_thread_sanitizer(tmp_path):
    if not _supports("g++", "-fsanitize=thread", tmp_path):
        pytest.skip("no ThreadSanitizer runtime")
    exe = _build_host(tmp_path, "thread")
    out = _run([str(exe), "3000", "8", str(tmp_path)], {"TSAN_OPTIONS": "halt_on_error=1 exitcode=66"})
    assert "ok" in out


def test_builder_under_address_sanitizer(tmp_path):
    if not _supports("g++", "-fsanitize=address,undefined", tmp_path):
        pytest.skip("no AddressSanitizer runtime")
    exe = _build_host(tmp_path, "address,undefined")
    out = _run([str(exe), "3000", "8", str(tmp_path)], {"ASAN_OPTIONS": "detect_leaks=1"})
    assert "ok" in out


def test_oracle_under_address_sanitizer(tmp_path):
    if not _supports("gcc", "-fsanitize=address,undefined", tmp_path):
        pytest.skip("no AddressSanitizer runtime")
    exe = tmp_path / "oracle_asan"
    subprocess.run(["gcc", "-std=c11", "-fsanitize=address,undefined", "-fno-sanitize-recover=undefined",
                    "-fno-omit-frame-pointer", "-g", "-O1", "-I", ORACLE, os.path.join(ORACLE, "hnsw_oracle.c"),
                    os.path.join(HERE, "oracle_sanitize_driver.c"), "-o", str(exe), "-lm"],
                   check=True, capture_output=True, timeout=300)
    out = _run([str(exe)], {"ASAN_OPTIONS": "detect_leaks=1"})
    assert "ok" in out
