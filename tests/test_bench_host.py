"""Host logic of `bench.py` that needs no GPU: the code key under which a profile's DRAM counters stay valid,
and the flop counts of the roofline line."""
import bench


def test_kernel_code_sha_ignores_comments_and_layout(tmp_path):
    base = "__global__ void k(float *x) {\n    x[0] += 1.0f;  // one\n}\n"
    comment = "// the kernel\n/* adds\n   one */\n__global__ void k(float *x) {\n  x[0] += 1.0f;\n}\n"
    code = "__global__ void k(float *x) {\n    x[0] += 2.0f;  // one\n}\n"
    paths = []
    for i, s in enumerate((base, comment, code)):
        p = tmp_path / ("k%d.cu" % i)
        p.write_text(s)
        paths.append(str(p))
    a, b, c = (bench.kernel_code_sha(p) for p in paths)
    assert a == b, "a comment or white-space edit must keep the key"
    assert a != c, "a code edit must change the key"
    assert len(a) == 12


def test_survey_flop_count_matches_quadruplet_count():
    # 16 FP32 flops per coupling term, 4|Q| terms per chain-sweep; |Q| of the N-mode comb by brute force
    for N in (4, 6, 16, 64):
        q = 0
        for a in range(N):
            for b in range(a + 1, N):
                for c in range(b + 1, N):
                    d = b + c - a
                    if c < d < N:
                        q += 1
        assert bench.count_quads(N) == q
        assert bench.survey_flops_per_chain_sweep(N) == 16.0 * 4 * q
    assert bench.count_quads(256) == 1373632
