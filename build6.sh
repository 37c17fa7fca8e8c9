#!/bin/bash
cd "$(dirname "$0")"
F="-gencode arch=compute_103a,code=sm_103a -O3 -lineinfo -std=c++17"
nvcc $F -o k6_cs kbench2.cu &
nvcc $F -DKV_PLAINST -o k6_plain kbench2.cu &
wait
ls k6_*
