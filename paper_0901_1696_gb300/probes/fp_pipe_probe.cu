// Arithmetic-pipe throughput probe behind the FP64 roofline peak used by the
// benchmark: dependent-chain-free DFMA, mma.sync.m8n8k4.f64 (DMMA) and FFMA
// streams on every SM (8 CTAs x 256 threads per SM), timed with CUDA events.
// Each thread writes one element of out[grid * block]; nothing else is read or
// written.  Build and run: python -m paper_0901_1696_gb300.build --probe
#include <cstdio>
#include <cuda_runtime.h>
#define CK(x) do{cudaError_t e=(x); if(e){printf("CUDA %s at %d\n",cudaGetErrorString(e),__LINE__); return 1;}}while(0)
template<int CH>
__global__ void dfma_probe(double* out, int iters, double a, double b){
  double acc[CH];
  for(int c=0;c<CH;++c) acc[c]=threadIdx.x*1e-9+c;
  for(int i=0;i<iters;++i){
#pragma unroll
    for(int c=0;c<CH;++c) acc[c]=fma(acc[c],a,b);
  }
  double s=0; for(int c=0;c<CH;++c) s+=acc[c];
  out[blockIdx.x*blockDim.x+threadIdx.x]=s;
}
template<int CH>
__global__ void ffma_probe(float* out, int iters, float a, float b){
  float acc[CH];
  for(int c=0;c<CH;++c) acc[c]=threadIdx.x*1e-6f+c;
  for(int i=0;i<iters;++i){
#pragma unroll
    for(int c=0;c<CH;++c) acc[c]=fmaf(acc[c],a,b);
  }
  float s=0; for(int c=0;c<CH;++c) s+=acc[c];
  out[blockIdx.x*blockDim.x+threadIdx.x]=s;
}
__global__ void dmma_probe(double* out, int iters){
  double a = 1.0 + threadIdx.x*1e-12, b = 0.999;
  double c0[2]={0,0}, c1[2]={0,0}, c2[2]={0,0}, c3[2]={0,0};
  for(int i=0;i<iters;++i){
#define MMA(c) asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};" : "+d"(c[0]), "+d"(c[1]) : "d"(a), "d"(b));
    MMA(c0) MMA(c1) MMA(c2) MMA(c3)
  }
  out[blockIdx.x*blockDim.x+threadIdx.x]=c0[0]+c1[1]+c2[0]+c3[1];
}
int main(){
  int dev=0; cudaDeviceProp p; CK(cudaGetDeviceProperties(&p,dev));
  int clk=0; cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, dev);
  printf("device %s SMs %d clock(kHz) %d cc %d.%d\n", p.name, p.multiProcessorCount, clk, p.major, p.minor);
  int sms=p.multiProcessorCount; int blocks=sms*8, threads=256; int n=blocks*threads;
  double* d; CK(cudaMalloc(&d, n*sizeof(double)));
  cudaEvent_t e0,e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
  float ms;
  for(int rep=0;rep<3;++rep){
    int iters=4096;
    dfma_probe<8><<<blocks,threads>>>(d,iters,0.9999999,1e-7); CK(cudaGetLastError());
    cudaEventRecord(e0); dfma_probe<8><<<blocks,threads>>>(d,iters,0.9999999,1e-7); cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
    cudaEventElapsedTime(&ms,e0,e1);
    printf("DFMA: %.3f TFLOP/s (%.3f ms)\n", 2.0*8*iters*(double)n/ms/1e9, ms);
    iters=2048;
    dmma_probe<<<blocks,threads>>>(d,iters); CK(cudaGetLastError());
    cudaEventRecord(e0); dmma_probe<<<blocks,threads>>>(d,iters); cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
    cudaEventElapsedTime(&ms,e0,e1);
    // per warp per mma: 8x8x4 = 256 FMA = 512 flop; 4 mma per iter
    double warps=(double)n/32;
    printf("DMMA m8n8k4: %.3f TFLOP/s (%.3f ms)\n", 512.0*4*iters*warps/ms/1e9, ms);
    iters=16384;
    ffma_probe<8><<<blocks,threads>>>((float*)d,iters,0.9999f,1e-4f); CK(cudaGetLastError());
    cudaEventRecord(e0); ffma_probe<8><<<blocks,threads>>>((float*)d,iters,0.9999f,1e-4f); cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
    cudaEventElapsedTime(&ms,e0,e1);
    printf("FFMA: %.3f TFLOP/s (%.3f ms)\n", 2.0*8*iters*(double)n/ms/1e9, ms);
  }
  CK(cudaFree(d));
  return 0;
}
