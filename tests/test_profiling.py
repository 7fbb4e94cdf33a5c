"""The launch-list summary used for the profiles (CPU only)."""
from paper_2508_18468_gb300 import profiling


def test_summary_groups_kernels_and_shares(tmp_path, capsys):
    p = tmp_path / "l.csv"
    hdr = '"ID","Kernel Name","Metric Name","Metric Unit","Metric Value"\n'
    rows = ['"0","void tc::tc_gemm_kernel<256, 0, 1>(CUtensorMap_st, Params)","gpu__time_duration.sum","ms","3.0"\n',
            '"1","chol_inv_leaf_kernel(const cplx<float> *, int)","gpu__time_duration.sum","us","500"\n',
            '"2","chol_inv_leaf_kernel(const cplx<float> *, int)","gpu__time_duration.sum","us","500"\n',
            '"3","chol_inv_leaf_kernel(const cplx<float> *, int)","dram__bytes_read.sum","byte","7"\n']
    p.write_text("==PROF== noise\n" + hdr + "".join(rows))
    profiling.summary(str(p))
    out = capsys.readouterr().out.splitlines()
    assert out[0] == "launches 3, total 4.0 ms"
    assert "75.0%" in out[2] and "tc_gemm_kernel<256, 0, 1>" in out[2]
    assert out[3].split()[:3] == ["2", "1.00", "25.0%"] and out[3].endswith("chol_inv_leaf_kernel")
